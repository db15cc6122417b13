// m1_spectrum_large.cu -- rows a3 + a4 of the hot path for sketch sizes above one
// CTA's shared memory (method 1, m = 2^15 .. 2^16, networks without open legs).
//
// a3: each sketch x (m reals, taken as m complex values with zero imaginary part)
// is transformed by the four-step split m = N1 N2, n = N2 n1 + n2:
//   pass 1: for blocks of columns n2, the N1-point DFTs over n1 in shared memory
//           (columns interleaved, so both the global reads and the butterflies
//           are conflict-free), times W_m^{n2 k1}, stored row-major to a global
//           scratch S[k1][n2];
//   pass 2: for blocks of rows k1, the N2-point DFTs over n2 in shared memory,
//           written back in place: S then holds (F x)(k1 + N1 k2) at row k1,
//           column bitrev(k2).
// Every sketch of a (network, rep) lands in the same permutation of the bins,
// which is all the product below needs.
// a4: y_r = (1/m) sum_j Re prod_k (F x_k)(j) over the full spectrum, one CTA per
// (network, rep, block of bins); the running product at each bin is kept as a
// mantissa in [0.5, 1) and a power-of-two exponent, and the sum is taken in FP64.
#include "fft.cuh"
#include "kernels.cuh"

namespace tnsk {

namespace {
template <typename T>
__host__ __device__ constexpr int large_fft_capacity() {  // complex values per pass: 128 KiB of shared memory
    return (int)((128 * 1024) / sizeof(Cplx<T>));
}
}  // namespace

template <typename T>
__global__ void __launch_bounds__(512) m1_fft_large_kernel(const M1Tensor* __restrict__ tens,
                                                           const M1Net* __restrict__ nets,
                                                           const int4* __restrict__ items, const T* __restrict__ xs,
                                                           const Cplx<T>* const* __restrict__ tws,
                                                           Cplx<T>* __restrict__ lspec) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cplx<T>* sm = reinterpret_cast<Cplx<T>*>(smem_raw);
    constexpr int C = large_fft_capacity<T>();
    const int4 it = items[blockIdx.x];  // (network, rep, sketch)
    const M1Net& N = nets[it.x];
    const int L = N.log2m;
    const int64_t m = N.m, half_m = m >> 1;
    const int L1 = L / 2, L2 = L - L1;
    const int N1 = 1 << L1, N2 = 1 << L2;
    const T* x = xs + N.x_off + (int64_t)it.y * N.X + tens[N.t0 + it.z].xoff;
    Cplx<T>* S = lspec + N.lspec_off + ((int64_t)it.y * N.p + it.z) * m;
    const Cplx<T>* __restrict__ twm = tws[L];  // exp(-2 pi i k / m), k < m / 2
    // ---- pass 1: columns
    int lb1 = L2;
    while ((1 << lb1) > C / N1) --lb1;
    const int B1 = 1 << lb1;
    for (int j0 = 0; j0 < N2; j0 += B1) {
        for (int idx = threadIdx.x; idx < (B1 << L1); idx += blockDim.x) {
            const int n1 = idx >> lb1, c = idx & (B1 - 1);
            sm[idx] = {x[(int64_t)n1 * N2 + j0 + c], T(0)};  // element n1 of column c at n1 * B1 + c
        }
        __syncthreads();
        block_fft_dif_interleaved(sm, lb1, L1, tws[L1 + 1]);
        for (int idx = threadIdx.x; idx < (B1 << L1); idx += blockDim.x) {
            const int k1 = idx >> lb1, c = idx & (B1 - 1);
            const int64_t n2 = j0 + c;
            const Cplx<T> a = sm[((int64_t)bitrev(k1, L1) << lb1) + c];
            const int64_t e = (n2 * k1) & (m - 1);
            const Cplx<T> w = e < half_m ? twm[e] : Cplx<T>{-twm[e - half_m].x, -twm[e - half_m].y};
            S[(int64_t)k1 * N2 + n2] = cmul(a, w);
        }
        __syncthreads();
    }
    // ---- pass 2: rows (this CTA's own pass-1 stores, ordered by the barriers)
    int lb2 = L1;
    while ((1 << lb2) > C / N2) --lb2;
    const int B2 = 1 << lb2;
    for (int k0 = 0; k0 < N1; k0 += B2) {
        Cplx<T>* rows = S + (int64_t)k0 * N2;
        for (int idx = threadIdx.x; idx < (B2 << L2); idx += blockDim.x) sm[idx] = rows[idx];
        __syncthreads();
        block_fft_dif(sm, B2, L2, tws[L2 + 1]);
        for (int idx = threadIdx.x; idx < (B2 << L2); idx += blockDim.x) rows[idx] = sm[idx];
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(256) m1_spec_product_kernel(const M1Net* __restrict__ nets,
                                                              const int4* __restrict__ items,
                                                              const Cplx<T>* __restrict__ lspec,
                                                              double* __restrict__ yrep) {
    __shared__ double red[32], rab[32];
    const int4 it = items[blockIdx.x];  // (network, rep, first bin, bins)
    const M1Net& N = nets[it.x];
    const int64_t m = N.m;
    const Cplx<T>* base = lspec + N.lspec_off + (int64_t)it.y * N.p * m;
    double acc = 0.0, aab = 0.0;  // the sum and the magnitude sum, as sum (|Re| + |Im|) (FP64 criterion)
    for (int64_t j = it.z + threadIdx.x; j < (int64_t)it.z + it.w; j += blockDim.x) {
        Cplx<T> P = {T(1), T(0)};
        int E = 0;  // the product is P 2^E
        for (int t = 0; t < N.p; ++t) {
            P = cmul(P, base[(int64_t)t * m + j]);
            const T mx = fmax(fabs(P.x), fabs(P.y));
            if (mx > T(0) && isfinite(mx)) {
                int e;
                frexp(mx, &e);
                P.x = ldexp(P.x, -e);
                P.y = ldexp(P.y, -e);
                E += e;
            }
        }
        acc += ldexp((double)P.x, E);
        aab += ldexp((double)(fabs(P.x) + fabs(P.y)), E);
    }
#pragma unroll
    for (int sft = 16; sft > 0; sft >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, sft);
        aab += __shfl_xor_sync(0xffffffffu, aab, sft);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[warp] = acc;
        rab[warp] = aab;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0, ta = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t += red[w];
            ta += rab[w];
        }
        atomicAdd(&yrep[N.y_off + it.y], t / (double)m);
        atomicAdd(&yrep[N.yabs_off + it.y], ta / (double)m);
    }
}

cudaError_t launch_m1_large(const M1Tensor* d_tens, const M1Net* d_nets, const int4* d_fft_items, int n_fft,
                            const int4* d_prod_items, int n_prod, const void* d_xs, const void* const* d_tws,
                            void* d_lspec, double* d_yrep, bool fp64, cudaStream_t s) {
    if (n_fft <= 0) return cudaSuccess;
    const int smem = 128 * 1024;
    if (fp64) {
        auto kf = m1_fft_large_kernel<double>;
        cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        kf<<<n_fft, 512, smem, s>>>(d_tens, d_nets, d_fft_items, (const double*)d_xs,
                                     (const Cplx<double>* const*)d_tws, (Cplx<double>*)d_lspec);
        m1_spec_product_kernel<double><<<n_prod, 256, 0, s>>>(d_nets, d_prod_items, (const Cplx<double>*)d_lspec,
                                                              d_yrep);
    } else {
        auto kf = m1_fft_large_kernel<float>;
        cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        kf<<<n_fft, 512, smem, s>>>(d_tens, d_nets, d_fft_items, (const float*)d_xs,
                                     (const Cplx<float>* const*)d_tws, (Cplx<float>*)d_lspec);
        m1_spec_product_kernel<float><<<n_prod, 256, 0, s>>>(d_nets, d_prod_items, (const Cplx<float>*)d_lspec,
                                                             d_yrep);
    }
    return cudaGetLastError();
}

}  // namespace tnsk
