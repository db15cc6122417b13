// fft.cuh -- block-cooperative shared-memory FFTs used by both estimators.
//
// A real sketch x of length m = 2M is transformed as M complex values
// z[n] = x[2n] + i x[2n+1] by an in-place radix-2 decimation-in-frequency FFT
// (output in bit-reversed order), then unpacked to the half spectrum
// X[k], k = 0..M, of the unnormalised DFT F_{jk} = exp(-2 pi i jk/m) (Sec. 2).
// The estimators only need products of spectra at equal frequencies and their
// sum, so the bit-reversed order is never undone for them.
#pragma once

#include "common.cuh"

namespace tnsk {

template <typename T>
__device__ __forceinline__ Cplx<T> cmul(Cplx<T> a, Cplx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ Cplx<T> cadd(Cplx<T> a, Cplx<T> b) {
    return {a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ Cplx<T> csub(Cplx<T> a, Cplx<T> b) {
    return {a.x - b.x, a.y - b.y};
}
template <typename T>
__device__ __forceinline__ Cplx<T> cconj(Cplx<T> a) {
    return {a.x, -a.y};
}

__device__ __forceinline__ int bitrev(int k, int log2M) {
    return log2M == 0 ? 0 : (int)(__brev((unsigned)k) >> (32 - log2M));
}

// In-place DIF FFT of nb consecutive length-M complex arrays in shared memory.
// tw[k] = exp(-2 pi i k / (2M)), k < M (the twiddles of the real length-2M
// transform; W_M^j = tw[2j]). Natural order in, bit-reversed order out.
// Must be called by all threads of the block; ends with __syncthreads().
template <typename T>
__device__ void block_fft_dif(Cplx<T>* z, int nb, int log2M, const Cplx<T>* __restrict__ tw) {
    const int M = 1 << log2M;
    if (log2M == 0) {
        __syncthreads();
        return;
    }
    const int lhb = log2M - 1;  // log2 of butterflies per array
    const int total = nb << lhb;
    for (int s = 0; s < log2M; ++s) {
        const int lhalf = log2M - s - 1;
        const int half = 1 << lhalf;
        const int tstride = 1 << (s + 1);
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int b = t >> lhb;
            const int u = t & ((1 << lhb) - 1);
            const int grp = u >> lhalf;
            const int j = u & (half - 1);
            const int i0 = (b << log2M) + (grp << (lhalf + 1)) + j;
            const int i1 = i0 + half;
            Cplx<T> a = z[i0], c = z[i1];
            z[i0] = cadd(a, c);
            Cplx<T> w = tw[j * tstride];
            z[i1] = cmul(csub(a, c), w);
        }
        __syncthreads();
    }
    (void)M;
}

// The same DIF FFT on nb arrays interleaved element by element: element i of
// array b sits at z[i * nb + b] (nb a power of two). Consecutive threads take the
// same butterfly of consecutive arrays, so shared-memory accesses are
// conflict-free; this is the layout of a block of columns of a row-major matrix.
// Natural order in, bit-reversed order out. Ends with __syncthreads().
template <typename T>
__device__ void block_fft_dif_interleaved(Cplx<T>* z, int log2nb, int log2M, const Cplx<T>* __restrict__ tw) {
    if (log2M == 0) {
        __syncthreads();
        return;
    }
    const int nb = 1 << log2nb;
    const int total = 1 << (log2nb + log2M - 1);  // butterflies per stage
    for (int s = 0; s < log2M; ++s) {
        const int lhalf = log2M - s - 1;
        const int half = 1 << lhalf;
        const int tstride = 1 << (s + 1);
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int b = t & (nb - 1);
            const int u = t >> log2nb;
            const int grp = u >> lhalf;
            const int j = u & (half - 1);
            const int i0 = (grp << (lhalf + 1)) + j;
            Cplx<T>* p0 = z + ((size_t)i0 << log2nb) + b;
            Cplx<T>* p1 = p0 + ((size_t)half << log2nb);
            const Cplx<T> a = *p0, c = *p1;
            *p0 = cadd(a, c);
            *p1 = cmul(csub(a, c), tw[j * tstride]);
        }
        __syncthreads();
    }
}

// Padded shared-memory layout for the fused transform below: element i at
// i + i / 32, so that the strided accesses of its last passes spread over the banks.
__device__ __forceinline__ int pidx(int i) { return i + (i >> 5); }

// A consecutive radix-2 DIF stages s .. s + A - 1 of a length-M transform (padded
// layout) in one pass: each thread loads the 2^A points i = base + sum_t b_t h_t
// (h_t = M >> (s + 1 + t), base free of those bits), applies the A stages' butterflies
// in registers with the same twiddles as block_fft_dif (stage s + t: W at index
// (i mod h_t) << (s + t + 1) of the length-2M table) and stores them back, so the
// result equals A separate radix-2 stages. Ends with __syncthreads().
template <typename T, int A>
__device__ __forceinline__ void fft_pass(Cplx<T>* z, int log2M, int s, const Cplx<T>* __restrict__ tw) {
    constexpr int P = 1 << A;
    const int lh0 = log2M - s - 1;  // log2 h_0
    const int lhl = lh0 - (A - 1);  // log2 h_{A-1}
    const int ngroups = 1 << (log2M - A);
    for (int g = threadIdx.x; g < ngroups; g += blockDim.x) {
        const int jl = g & ((1 << lhl) - 1);
        const int base = ((g >> lhl) << (lh0 + 1)) + jl;
        int at[P];
        Cplx<T> v[P];
#pragma unroll
        for (int q = 0; q < P; ++q) {
            int off = 0;
#pragma unroll
            for (int t = 0; t < A; ++t)
                if ((q >> (A - 1 - t)) & 1) off += 1 << (lh0 - t);
            at[q] = pidx(base + off);
            v[q] = z[at[q]];
        }
#pragma unroll
        for (int t = 0; t < A; ++t) {
            const int bit = 1 << (A - 1 - t);
#pragma unroll
            for (int q = 0; q < P; ++q) {
                if (q & bit) continue;
                int j = jl;  // the pair's index within its half-group at stage s + t
#pragma unroll
                for (int u = t + 1; u < A; ++u)
                    if ((q >> (A - 1 - u)) & 1) j += 1 << (lh0 - u);
                const Cplx<T> a = v[q], c = v[q | bit];
                v[q] = cadd(a, c);
                v[q | bit] = cmul(csub(a, c), tw[j << (s + t + 1)]);
            }
        }
#pragma unroll
        for (int q = 0; q < P; ++q) z[at[q]] = v[q];
    }
    __syncthreads();
}

// The DIF FFT of one length-M array in the padded layout, three stages per pass
// (then a pass of two or one): natural order in, bit-reversed order out, the same
// values as block_fft_dif. tw as there (may point to global memory).
template <typename T>
__device__ void block_fft_dif_fused(Cplx<T>* z, int log2M, const Cplx<T>* __restrict__ tw) {
    int s = 0;
    for (; log2M - s >= 3; s += 3) fft_pass<T, 3>(z, log2M, s, tw);
    if (log2M - s == 2) fft_pass<T, 2>(z, log2M, s, tw);
    else if (log2M - s == 1) fft_pass<T, 1>(z, log2M, s, tw);
    else __syncthreads();
}

// Half-spectrum bin k (0..M) of the real sequence whose packed transform Z sits
// bit-reversed in z in the padded layout.
template <typename T>
__device__ __forceinline__ Cplx<T> unpack_bin_padded(const Cplx<T>* z, int k, int log2M,
                                                     const Cplx<T>* __restrict__ tw) {
    const int M = 1 << log2M;
    Cplx<T> zk = z[pidx(bitrev(k & (M - 1), log2M))];
    Cplx<T> zc = cconj(z[pidx(bitrev((M - k) & (M - 1), log2M))]);
    Cplx<T> e = {(zk.x + zc.x) * T(0.5), (zk.y + zc.y) * T(0.5)};
    Cplx<T> d = csub(zk, zc);
    Cplx<T> o = {d.y * T(0.5), -d.x * T(0.5)};  // (Zk - conj Z_{M-k}) / (2i)
    Cplx<T> w = (k < M) ? tw[k] : Cplx<T>{T(-1), T(0)};
    return cadd(e, cmul(w, o));
}

// Half-spectrum bin k (0..M) of the real sequence whose packed transform Z sits
// bit-reversed in z (one array of length M).
template <typename T>
__device__ __forceinline__ Cplx<T> unpack_bin(const Cplx<T>* z, int k, int log2M, const Cplx<T>* __restrict__ tw) {
    const int M = 1 << log2M;
    Cplx<T> zk = z[bitrev(k & (M - 1), log2M)];
    Cplx<T> zc = cconj(z[bitrev((M - k) & (M - 1), log2M)]);
    Cplx<T> e = {(zk.x + zc.x) * T(0.5), (zk.y + zc.y) * T(0.5)};
    Cplx<T> d = csub(zk, zc);
    Cplx<T> o = {d.y * T(0.5), -d.x * T(0.5)};  // (Zk - conj Z_{M-k}) / (2i)
    Cplx<T> w = (k < M) ? tw[k] : Cplx<T>{T(-1), T(0)};
    return cadd(e, cmul(w, o));
}

}  // namespace tnsk
