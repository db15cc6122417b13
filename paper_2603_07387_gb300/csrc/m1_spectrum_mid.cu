// m1_spectrum_mid.cu -- rows a3 + a4 of the hot path for closed networks at
// m = 2^11 .. 2^14 (method 1), one CTA per sketch instead of one per (network, rep).
//
// a3: each sketch x (m reals) is transformed as M = m/2 packed complex values
// z[n] = x[2n] + i x[2n+1] by the shared-memory DIF FFT with three radix-2 stages per
// pass in registers (fft.cuh, padded layout) and unpacked to
// its half spectrum X[k], k = 0..M, of the unnormalised DFT (Sec. 2), written to a
// global scratch [R][p][M + 1] per network. Every sketch of a (network, rep) lands in
// the same bin order, which is all the product needs.
// a4: y_r = (1/m) sum_j Re prod_k (F x_k)(j) over the full spectrum; the full
// spectrum is Hermitian, so sum_j = P[0] + P[M] + 2 sum_{0<k<M} Re P[k]. One CTA per
// (network, rep, block of bins); the running product at each bin is kept as a
// mantissa in [0.5, 1) times a power of two, and the sum is taken in FP64.
// With R x p CTAs for the transforms the work spreads over the whole GPU even for
// one network and few reps, where one CTA per (network, rep) would leave most SMs idle.
#include "fft.cuh"
#include "kernels.cuh"

namespace tnsk {

template <typename T>
__global__ void __launch_bounds__(512) m1_fft_mid_kernel(const M1Tensor* __restrict__ tens,
                                                         const M1Net* __restrict__ nets,
                                                         const int4* __restrict__ items, const T* __restrict__ xs,
                                                         const Cplx<T>* const* __restrict__ tws,
                                                         Cplx<T>* __restrict__ lspec) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cplx<T>* z = reinterpret_cast<Cplx<T>*>(smem_raw);
    const int4 it = items[blockIdx.x];  // (network, rep, sketch)
    const M1Net& N = nets[it.x];
    const int log2M = N.log2m - 1;
    const int M = 1 << log2M;
    const int64_t K = (int64_t)M + 1;
    const T* x = xs + N.x_off + (int64_t)it.y * N.X + tens[N.t0 + it.z].xoff;
    Cplx<T>* X = lspec + N.lspec_off + ((int64_t)it.y * N.p + it.z) * K;
    const Cplx<T>* __restrict__ tw = tws[N.log2m];  // exp(-2 pi i k / m), k < M
    for (int n = threadIdx.x; n < M; n += blockDim.x) z[pidx(n)] = {x[2 * n], x[2 * n + 1]};
    __syncthreads();
    block_fft_dif_fused(z, log2M, tw);
    for (int k = threadIdx.x; k <= M; k += blockDim.x) X[k] = unpack_bin_padded(z, k, log2M, tw);
}

template <typename T>
__global__ void __launch_bounds__(256) m1_spec_product_half_kernel(const M1Net* __restrict__ nets,
                                                                   const int4* __restrict__ items,
                                                                   const Cplx<T>* __restrict__ lspec,
                                                                   double* __restrict__ yrep) {
    __shared__ double red[32], rab[32];
    const int4 it = items[blockIdx.x];  // (network, rep, first bin, bins)
    const M1Net& N = nets[it.x];
    const int64_t M = N.m >> 1, K = M + 1;
    const Cplx<T>* base = lspec + N.lspec_off + (int64_t)it.y * N.p * K;
    double acc = 0.0, aab = 0.0;  // the sum and the magnitude sum, as sum (|Re| + |Im|) (FP64 criterion)
    for (int64_t j = it.z + threadIdx.x; j < (int64_t)it.z + it.w; j += blockDim.x) {
        Cplx<T> P = {T(1), T(0)};
        int E = 0;  // the product is P 2^E
        for (int t = 0; t < N.p; ++t) {
            P = cmul(P, base[(int64_t)t * K + j]);
            const T mx = fmax(fabs(P.x), fabs(P.y));
            if (mx > T(0) && isfinite(mx)) {
                int e;
                frexp(mx, &e);
                P.x = ldexp(P.x, -e);
                P.y = ldexp(P.y, -e);
                E += e;
            }
        }
        const double w = (j == 0 || j == M) ? 1.0 : 2.0;
        acc += w * ldexp((double)P.x, E);
        aab += w * ldexp((double)(fabs(P.x) + fabs(P.y)), E);
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
        atomicAdd(&yrep[N.y_off + it.y], t / (double)N.m);
        atomicAdd(&yrep[N.yabs_off + it.y], ta / (double)N.m);
    }
}

size_t m1_mid_smem(int max_log2m, bool fp64) {
    const size_t M = (size_t)1 << (max_log2m - 1);
    return (M + M / 32) * (fp64 ? 16 : 8);  // the padded layout
}

cudaError_t launch_m1_mid(const M1Tensor* d_tens, const M1Net* d_nets, const int4* d_fft_items, int n_fft,
                          const int4* d_prod_items, int n_prod, int max_log2m, const void* d_xs,
                          const void* const* d_tws, void* d_lspec, double* d_yrep, bool fp64, cudaStream_t s) {
    if (n_fft <= 0) return cudaSuccess;
    const int smem = (int)m1_mid_smem(max_log2m, fp64);
    if (fp64) {
        auto kf = m1_fft_mid_kernel<double>;
        cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        kf<<<n_fft, 512, smem, s>>>(d_tens, d_nets, d_fft_items, (const double*)d_xs,
                                     (const Cplx<double>* const*)d_tws, (Cplx<double>*)d_lspec);
        m1_spec_product_half_kernel<double><<<n_prod, 256, 0, s>>>(d_nets, d_prod_items,
                                                                   (const Cplx<double>*)d_lspec, d_yrep);
    } else {
        auto kf = m1_fft_mid_kernel<float>;
        cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        kf<<<n_fft, 512, smem, s>>>(d_tens, d_nets, d_fft_items, (const float*)d_xs,
                                     (const Cplx<float>* const*)d_tws, (Cplx<float>*)d_lspec);
        m1_spec_product_half_kernel<float><<<n_prod, 256, 0, s>>>(d_nets, d_prod_items, (const Cplx<float>*)d_lspec,
                                                                  d_yrep);
    }
    return cudaGetLastError();
}

}  // namespace tnsk
