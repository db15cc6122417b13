// m1_spectrum_large.cu -- rows a3 + a4 of the hot path for sketch sizes above one
// CTA's shared memory (method 1, m = 2^15 .. 2^16 in FP32, 2^14 .. 2^16 in FP64,
// networks without open legs).
//
// a3: each sketch x (m reals) is transformed as M = m/2 packed complex values
// z[n] = x[2n] + i x[2n+1] by the four-step split M = N1 N2, n = N2 n1 + n2:
//   pass 1 (one CTA per sketch): for blocks of columns n2, the N1-point DFTs over n1
//           in shared memory (columns interleaved, so both the global reads and the
//           butterflies are conflict-free), times W_M^{n2 k1}, stored row-major to a
//           global scratch S[k1][n2] (M complex values per sketch);
//   pass 2 (one CTA per network, rep and pair of rows {k1, N1 - k1}): the rows of
//           every sketch of the rep go through the N2-point DFT over n2 in shared
//           memory, giving Z(k1 + N1 k2) at column bitrev(k2); the real sketch's
//           spectrum follows by the unpack X(k) = (Z(k) + conj Z(M-k)) / 2 +
//           W_m^k (Z(k) - conj Z(M-k)) / (2i), and M - k lies in the partner row
//           N1 - k1 (row 0 and row N1/2 are their own partners), so the pair of rows
//           holds every bin it needs.
// a4: in the same pass-2 CTA, the running product over the sketches at each of its
// bins is kept as a mantissa in [0.5, 1) times a power of two, and
// y_r = (1/m) sum_j Re prod_k (F x_k)(j) = (1/m) (P(0) + P(M) + 2 sum_{0<k<M} Re P(k))
// is summed in FP64 over the CTAs of the rep (the Nyquist bin P(M) comes with k = 0).
// The scratch holds half the values a complex transform of x would, and the
// spectra are read once, by the CTA that multiplies them.
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
    const int L = N.log2m, LM = L - 1;
    const int64_t M = (int64_t)1 << LM;
    const int L1 = LM / 2, L2 = LM - L1;
    const int N1 = 1 << L1, N2 = 1 << L2;
    const T* x = xs + N.x_off + (int64_t)it.y * N.X + tens[N.t0 + it.z].xoff;
    Cplx<T>* S = lspec + N.lspec_off + ((int64_t)it.y * N.p + it.z) * M;
    const Cplx<T>* __restrict__ twm = tws[L];  // exp(-2 pi i k / m), k < M
    int lb1 = L2;
    while ((1 << lb1) > C / N1) --lb1;
    const int B1 = 1 << lb1;
    for (int j0 = 0; j0 < N2; j0 += B1) {
        for (int idx = threadIdx.x; idx < (B1 << L1); idx += blockDim.x) {
            const int n1 = idx >> lb1, c = idx & (B1 - 1);
            const int64_t n = (int64_t)n1 * N2 + j0 + c;  // packed element n of column c at n1 * B1 + c
            sm[idx] = reinterpret_cast<const Cplx<T>*>(x)[n];  // (x[2n], x[2n+1]); sketches are 16-byte aligned
        }
        __syncthreads();
        block_fft_dif_interleaved(sm, lb1, L1, tws[L1 + 1]);
        for (int idx = threadIdx.x; idx < (B1 << L1); idx += blockDim.x) {
            const int k1 = idx >> lb1, c = idx & (B1 - 1);
            const int64_t n2 = j0 + c;
            const Cplx<T> a = sm[((int64_t)bitrev(k1, L1) << lb1) + c];
            // W_M^e = W_m^{2e}, 2e mod m taken from the table of the first half
            const int64_t e2 = (2 * ((n2 * k1) & (M - 1))) & (2 * M - 1);
            const Cplx<T> w = e2 < M ? twm[e2] : Cplx<T>{-twm[e2 - M].x, -twm[e2 - M].y};
            S[(int64_t)k1 * N2 + n2] = cmul(a, w);
        }
        __syncthreads();
    }
}

// Pass 2 and the product: one CTA per (network, rep, row k1 in [0, N1/2]); rows k1 and
// N1 - k1 (one row when k1 is 0 or N1/2) of every sketch, G sketches at a time in
// shared memory. Each thread keeps the running products of its bins in registers.
template <typename T>
__global__ void __launch_bounds__(256) m1_large_rows_kernel(const M1Net* __restrict__ nets,
                                                            const int4* __restrict__ items,
                                                            const Cplx<T>* const* __restrict__ tws,
                                                            const Cplx<T>* __restrict__ lspec,
                                                            double* __restrict__ yrep) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cplx<T>* sz = reinterpret_cast<Cplx<T>*>(smem_raw);  // [g][nrow][N2]
    constexpr int kMaxB = 4;  // bins per thread: 2 N2 <= 1024 with 256 threads
    __shared__ double red[8], rab[8];
    const int4 it = items[blockIdx.x];  // (network, rep, k1, sketches per group)
    const M1Net& N = nets[it.x];
    const int L = N.log2m, LM = L - 1;
    const int64_t M = (int64_t)1 << LM;
    const int L1 = LM / 2, L2 = LM - L1;
    const int N1 = 1 << L1, N2 = 1 << L2;
    const int k1 = it.z;
    const int k1b = (k1 == 0 || 2 * k1 == N1) ? k1 : N1 - k1;
    const int nrow = k1b == k1 ? 1 : 2;
    const int G = it.w;
    const Cplx<T>* __restrict__ twm = tws[L];       // exp(-2 pi i k / m), k < M
    const Cplx<T>* __restrict__ tw2 = tws[L2 + 1];  // the N2-point transform's
    const Cplx<T>* base = lspec + N.lspec_off + (int64_t)it.y * N.p * M;
    const int nb = nrow * N2;  // bins of this CTA
    // per owned bin: its half-spectrum index k, its slot, its partner's slot
    int kk[kMaxB], sl[kMaxB], sp[kMaxB];
    Cplx<T> P[kMaxB];
    int E[kMaxB];
    Cplx<T> PN = {T(1), T(0)};  // the Nyquist bin M, kept by the thread holding k = 0
    int EN = 0;
#pragma unroll
    for (int s = 0; s < kMaxB; ++s) {
        const int b = threadIdx.x + s * blockDim.x;
        kk[s] = -1;
        P[s] = {T(1), T(0)};
        E[s] = 0;
        if (b < nb) {
            const int r = b >> L2, pos = b & (N2 - 1);
            const int64_t k = (int64_t)(r == 0 ? k1 : k1b) + (int64_t)N1 * bitrev(pos, L2);
            const int64_t kp = (M - k) & (M - 1);  // partner bin M - k (0 for k = 0)
            const int rp = (int)(kp & (N1 - 1)) == k1 ? 0 : 1;
            kk[s] = (int)k;
            sl[s] = b;
            sp[s] = rp * N2 + bitrev((int)(kp >> L1), L2);
        }
    }
    for (int t0 = 0; t0 < N.p; t0 += G) {
        const int g = min(G, N.p - t0);
        __syncthreads();  // the previous group's reads are done
        for (int idx = threadIdx.x; idx < g * nb; idx += blockDim.x) {
            const int j = idx / nb, b = idx - j * nb;
            const int r = b >> L2, n2 = b & (N2 - 1);
            sz[idx] = base[(int64_t)(t0 + j) * M + (int64_t)(r == 0 ? k1 : k1b) * N2 + n2];
        }
        __syncthreads();
        block_fft_dif(sz, g * nrow, L2, tw2);
#pragma unroll
        for (int s = 0; s < kMaxB; ++s) {
            if (kk[s] < 0) continue;
            const Cplx<T> w = twm[kk[s]];
            for (int j = 0; j < g; ++j) {
                const Cplx<T> zk = sz[j * nb + sl[s]];
                const Cplx<T> zc = cconj(sz[j * nb + sp[s]]);
                const Cplx<T> e = {(zk.x + zc.x) * T(0.5), (zk.y + zc.y) * T(0.5)};
                const Cplx<T> d = csub(zk, zc);
                const Cplx<T> o = {d.y * T(0.5), -d.x * T(0.5)};  // (Z(k) - conj Z(M-k)) / (2i)
                P[s] = cmul(P[s], cadd(e, cmul(w, o)));
                const T mx = fmax(fabs(P[s].x), fabs(P[s].y));
                if (mx > T(0) && isfinite(mx)) {
                    int ex;
                    frexp(mx, &ex);
                    P[s].x = ldexp(P[s].x, -ex);
                    P[s].y = ldexp(P[s].y, -ex);
                    E[s] += ex;
                }
                if (kk[s] == 0) {  // X(M) = Re Z(0) - Im Z(0)
                    PN = cmul(PN, Cplx<T>{zk.x - zk.y, T(0)});
                    const T mn = fabs(PN.x);
                    if (mn > T(0) && isfinite(mn)) {
                        int ex;
                        frexp(mn, &ex);
                        PN.x = ldexp(PN.x, -ex);
                        EN += ex;
                    }
                }
            }
        }
    }
    // sum_j Re P(j) over the full spectrum: weight 1 for bins 0 and M, 2 for 0 < k < M
    double acc = 0.0, aab = 0.0;
#pragma unroll
    for (int s = 0; s < kMaxB; ++s) {
        if (kk[s] < 0) continue;
        const double wt = kk[s] == 0 ? 1.0 : 2.0;
        acc += wt * ldexp((double)P[s].x, E[s]);
        aab += wt * ldexp((double)(fabs(P[s].x) + fabs(P[s].y)), E[s]);
        if (kk[s] == 0) {
            acc += ldexp((double)PN.x, EN);
            aab += ldexp((double)fabs(PN.x), EN);
        }
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
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            t += red[q];
            ta += rab[q];
        }
        atomicAdd(&yrep[N.y_off + it.y], t / (double)N.m);
        atomicAdd(&yrep[N.yabs_off + it.y], ta / (double)N.m);
    }
}

size_t m1_large_rows_smem(int log2m, int G, bool fp64) {
    const int LM = log2m - 1, L2 = LM - LM / 2;
    return (size_t)G * 2 * ((size_t)1 << L2) * (fp64 ? 16 : 8);
}

int m1_large_rows_group(int log2m, int p, bool fp64) {
    const size_t per = m1_large_rows_smem(log2m, 1, fp64);
    const int g = (int)((96 * 1024) / per);
    return std::max(1, std::min(p, g));
}

cudaError_t launch_m1_large(const M1Tensor* d_tens, const M1Net* d_nets, const int4* d_fft_items, int n_fft,
                            const int4* d_prod_items, int n_prod, size_t rows_smem, const void* d_xs,
                            const void* const* d_tws, void* d_lspec, double* d_yrep, bool fp64, cudaStream_t s) {
    if (n_fft <= 0) return cudaSuccess;
    const int smem = 128 * 1024;
    if (fp64) {
        auto kf = m1_fft_large_kernel<double>;
        cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        kf<<<n_fft, 512, smem, s>>>(d_tens, d_nets, d_fft_items, (const double*)d_xs,
                                     (const Cplx<double>* const*)d_tws, (Cplx<double>*)d_lspec);
        auto kr = m1_large_rows_kernel<double>;
        cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem);
        kr<<<n_prod, 256, rows_smem, s>>>(d_nets, d_prod_items, (const Cplx<double>* const*)d_tws,
                                          (const Cplx<double>*)d_lspec, d_yrep);
    } else {
        auto kf = m1_fft_large_kernel<float>;
        cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        kf<<<n_fft, 512, smem, s>>>(d_tens, d_nets, d_fft_items, (const float*)d_xs,
                                     (const Cplx<float>* const*)d_tws, (Cplx<float>*)d_lspec);
        auto kr = m1_large_rows_kernel<float>;
        cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem);
        kr<<<n_prod, 256, rows_smem, s>>>(d_nets, d_prod_items, (const Cplx<float>* const*)d_tws,
                                          (const Cplx<float>*)d_lspec, d_yrep);
    }
    return cudaGetLastError();
}

}  // namespace tnsk
