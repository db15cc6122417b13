// m1_spectrum_warp.cu -- rows a3 + a4 of the hot path for FP32 networks with
// 64 <= m <= 1024: one warp per (network, rep), every FFT held in registers.
//
// y_r = (1/m) sum_j prod_k (F x_k)(j) (Alg. 1, last line). A real sketch x of
// length m = 2M is transformed as z[n] = x[2n] + i x[2n+1] (M complex points)
// with the four-step split M = 32 J (J = 1..16 values per lane):
//   1. lane l holds z[l + 32 j], j < J, and takes the J-point DFT over j in
//      registers, then multiplies by W_M^{l k1};
//   2. a transpose through a per-warp shared buffer gives lane L = k1 G + g
//      (G = 32 / J lanes per k1) the values of lanes l = g + G i; a second
//      J-point DFT in registers, the twiddle W_32^{g k} and a G-point DFT across
//      the G lanes (shuffle butterflies) finish the 32-point DFTs over l.
// Lane L then holds Z[q], q = k1 + J k + J^2 c (c = bit reverse of g), for its
// J registers k. The half spectrum X[q] of x needs Z[M - q] too (the real-FFT
// unpack); that value sits in a lane and register known in closed form and
// comes over one shuffle per register. Products at equal frequencies and the
// final sum do not depend on where a bin sits, so the spectrum is never put
// back in order. As in the block kernel, each spectrum is scaled by 2^-e (e
// from its largest component) before it enters the running product, and the
// sum sum_j = X[0] + X[M] + 2 Re sum_{0<q<M} X[q] is taken in FP64.
// Tensors with open legs (one sketch per open index, Corollary "full-to-partial-
// tc") have their scaled spectra stored, in natural bin order with their
// exponents (the block kernel's layout); every output entry is then the sum over
// bins of the running product times one stored spectrum per open tensor.
#include "fft.cuh"
#include "kernels.cuh"

namespace tnsk {
namespace {

using C32 = Cplx<float>;

__host__ __device__ constexpr int brev_bits(int x, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b)
        if ((x >> b) & 1) r |= 1 << (bits - 1 - b);
    return r;
}

// v * exp(-2 pi i k / 16); k is a compile-time constant wherever this is used.
__device__ __forceinline__ C32 mul_w16(C32 v, int k) {
    constexpr float c1 = 0.92387953251128674f;  // cos(pi / 8)
    constexpr float s1 = 0.38268343236508977f;  // sin(pi / 8)
    constexpr float h = 0.70710678118654752f;   // cos(pi / 4)
    switch (k & 15) {
        case 0: return v;
        case 4: return {v.y, -v.x};
        case 8: return {-v.x, -v.y};
        case 12: return {-v.y, v.x};
        case 1: return cmul(v, C32{c1, -s1});
        case 2: return cmul(v, C32{h, -h});
        case 3: return cmul(v, C32{s1, -c1});
        case 5: return cmul(v, C32{-s1, -c1});
        case 6: return cmul(v, C32{-h, -h});
        case 7: return cmul(v, C32{-c1, -s1});
        case 9: return cmul(v, C32{-c1, s1});
        case 10: return cmul(v, C32{-h, h});
        case 11: return cmul(v, C32{-s1, c1});
        case 13: return cmul(v, C32{s1, c1});
        case 14: return cmul(v, C32{h, h});
        default: return cmul(v, C32{c1, s1});
    }
}

// In-register J-point DFT (J <= 16): radix-2 decimation in frequency, then the
// bit-reversal permutation as a renaming of registers. Natural order in and out.
template <int J>
__device__ __forceinline__ void dft_reg(C32 (&v)[J]) {
#pragma unroll
    for (int half = J / 2; half >= 1; half >>= 1) {
#pragma unroll
        for (int i0 = 0; i0 < J; i0 += 2 * half) {
#pragma unroll
            for (int j = 0; j < half; ++j) {
                const C32 a = v[i0 + j], b = v[i0 + j + half];
                v[i0 + j] = cadd(a, b);
                v[i0 + j + half] = mul_w16(csub(a, b), j * (16 / (2 * half)));  // W_{2 half}^j
            }
        }
    }
    constexpr int LB = J == 1 ? 0 : (J == 2 ? 1 : (J == 4 ? 2 : (J == 8 ? 3 : 4)));
    C32 t[J];
#pragma unroll
    for (int i = 0; i < J; ++i) t[i] = v[brev_bits(i, LB)];
#pragma unroll
    for (int i = 0; i < J; ++i) v[i] = t[i];
}

__device__ __forceinline__ C32 shfl_c(C32 v, int src) {
    return {__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}
__device__ __forceinline__ C32 shfl_xor_c(C32 v, int mask) {
    return {__shfl_xor_sync(0xffffffffu, v.x, mask), __shfl_xor_sync(0xffffffffu, v.y, mask)};
}

constexpr int kWarps = 8;

}  // namespace

template <int LOGJ>
__global__ void __launch_bounds__(kWarps * 32, 2)
    m1_spectrum_warp_kernel(const M1Tensor* __restrict__ tens, const M1Net* __restrict__ nets,
                            const OpenMode* __restrict__ opens, const int2* __restrict__ items, int n_items,
                            const float* __restrict__ xs, const C32* const* __restrict__ tws, C32* __restrict__ spec,
                            int* __restrict__ sexp, double* __restrict__ yrep) {
    constexpr int J = 1 << LOGJ, LOGG = 5 - LOGJ, G = 1 << LOGG;
    constexpr int M = 32 * J, m = 2 * M;
    constexpr int S = 32 + (G & 15);  // row stride of the transpose buffer: conflict-free both ways
    __shared__ C32 twA[J][32];        // W_M^{l k1}          (step 1, lane l)
    __shared__ C32 twB[J][32];        // W_32^{g k}          (step 2, lane L = k1 G + g)
    __shared__ C32 twC[J][32];        // W_m^q of the bin in (lane, register)
    __shared__ C32 buf[kWarps][J * S];
    const C32* __restrict__ tw = tws[LOGJ + 6];  // exp(-2 pi i k / m), k < M
    auto twm = [&](int e) -> C32 {
        e &= m - 1;
        return e < M ? tw[e] : C32{-tw[e - M].x, -tw[e - M].y};
    };
    for (int idx = threadIdx.x; idx < J * 32; idx += blockDim.x) {
        const int k = idx >> 5, L = idx & 31;
        const int g = L & (G - 1), k1 = L >> LOGG;
        twA[k][L] = twm(2 * L * k);
        twB[k][L] = twm(g * k * (m / 32));
        twC[k][L] = tw[k1 + J * k + J * J * brev_bits(g, LOGG)];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int item = blockIdx.x * kWarps + warp;
    if (item >= n_items) return;
    const int2 it = items[item];
    const M1Net& N = nets[it.x];
    const int r = it.y;
    const float* xr = xs + N.x_off + (int64_t)r * N.X;
    const int k1L = lane >> LOGG, gL = lane & (G - 1), cL = brev_bits(gL, LOGG);
    C32 wst[LOGG > 0 ? LOGG : 1];  // cross-lane butterfly twiddles W_{2h}^{g mod h}
#pragma unroll
    for (int s = 0; s < LOGG; ++s) {
        const int h = G >> (s + 1);
        wst[s] = twm((gL & (h - 1)) * (m / (2 * h)));
    }
    // partner lane of each register for the unpack: Z[M - q]
    const int src_hi = (J - k1L) * G + (G - 1 - gL);                           // k1 != 0
    const int src_k0 = cL == 0 ? lane : brev_bits((G - cL) & (G - 1), LOGG);    // k1 == 0, k == 0
    C32* wb = buf[warp];
    C32 P[J];
#pragma unroll
    for (int k = 0; k < J; ++k) P[k] = {1.f, 0.f};
    float PM = 1.f;  // bin M (real), kept by lane 0
    int E = 0;       // P holds 2^-E prod_k F x_k
    C32* Sb = spec + N.spec_off + (int64_t)r * N.spec_per_rep;
    int* Eb = sexp + N.exp_off + (int64_t)r * N.exp_per_rep;
    constexpr int K = M + 1;  // stored half spectrum: bins 0 .. M
    for (int t = 0; t < N.p; ++t) {
        const M1Tensor& Tk = tens[N.t0 + t];
        const int64_t nsk = Tk.soff < 0 ? 1 : Tk.O;
        for (int64_t os = 0; os < nsk; ++os) {
            const C32* z = reinterpret_cast<const C32*>(xr + Tk.xoff + os * m);  // 8-byte aligned
            C32 v[J];
#pragma unroll
            for (int j = 0; j < J; ++j) v[j] = z[lane + 32 * j];
            dft_reg<J>(v);
#pragma unroll
            for (int k = 0; k < J; ++k) wb[k * S + lane] = cmul(v[k], twA[k][lane]);
            __syncwarp();
#pragma unroll
            for (int i = 0; i < J; ++i) v[i] = wb[k1L * S + gL + G * i];
            __syncwarp();
            dft_reg<J>(v);
#pragma unroll
            for (int k = 0; k < J; ++k) v[k] = cmul(v[k], twB[k][lane]);
#pragma unroll
            for (int s = 0; s < LOGG; ++s) {
                const int h = G >> (s + 1);
                const bool up = (gL & h) != 0;
#pragma unroll
                for (int k = 0; k < J; ++k) {
                    const C32 o = shfl_xor_c(v[k], h);
                    v[k] = up ? cmul(csub(o, v[k]), wst[s]) : cadd(v[k], o);
                }
            }
            // real-FFT unpack: X[q] = (Z[q] + conj Z[M-q]) / 2 + W_m^q (Z[q] - conj Z[M-q]) / (2i)
            C32 X[J];
#pragma unroll
            for (int k = 0; k < J; ++k) {
                const C32 send = k1L == 0 ? v[(J - k) & (J - 1)] : v[J - 1 - k];
                const int src = k1L != 0 ? src_hi : (k != 0 ? G - 1 - gL : src_k0);
                const C32 zc = cconj(shfl_c(send, src));
                const C32 zk = v[k];
                const C32 e = {(zk.x + zc.x) * 0.5f, (zk.y + zc.y) * 0.5f};
                const C32 d = csub(zk, zc);
                const C32 o = {d.y * 0.5f, -d.x * 0.5f};
                X[k] = cadd(e, cmul(o, twC[k][lane]));
            }
            const float XM = v[0].x - v[0].y;  // meaningful in lane 0 only (q = 0 there)
            float mx = lane == 0 ? fabsf(XM) : 0.f;
#pragma unroll
            for (int k = 0; k < J; ++k) mx = fmaxf(mx, fmaxf(fabsf(X[k].x), fabsf(X[k].y)));
            // non-negative floats order like their bit patterns
            const unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
            int e = 0;
            if (mb != 0u) frexpf(__uint_as_float(mb), &e);
            const float sc = ldexpf(1.f, -e);
            if (Tk.soff < 0) {
#pragma unroll
                for (int k = 0; k < J; ++k) P[k] = cmul(P[k], C32{X[k].x * sc, X[k].y * sc});
                PM *= XM * sc;
                E += e;
            } else {  // an open index of an open tensor: keep its scaled spectrum
                C32* dst = Sb + Tk.soff + os * K;
#pragma unroll
                for (int k = 0; k < J; ++k) dst[k1L + J * k + J * J * cL] = C32{X[k].x * sc, X[k].y * sc};
                if (lane == 0) {
                    dst[M] = C32{XM * sc, 0.f};
                    Eb[Tk.eoff + os] = e;
                }
            }
        }
    }
    double* yr = yrep + N.y_off + (int64_t)r * N.O;
    if (N.n_ot == 0) {
        double acc = lane == 0 ? (double)PM : 0.0;
        // the magnitude sum for the FP64 criterion, as sum (|Re| + |Im|): FP32 suffices
        float aab = lane == 0 ? fabsf(PM) : 0.f;
#pragma unroll
        for (int k = 0; k < J; ++k) {
            const int q = k1L + J * k + J * J * cL;
            acc += (q == 0 ? 1.0 : 2.0) * (double)P[k].x;
            aab += (q == 0 ? 1.f : 2.f) * (fabsf(P[k].x) + fabsf(P[k].y));
        }
#pragma unroll
        for (int sft = 16; sft > 0; sft >>= 1) {
            acc += __shfl_xor_sync(0xffffffffu, acc, sft);
            aab += __shfl_xor_sync(0xffffffffu, aab, sft);
        }
        if (lane == 0) {
            yr[0] = ldexp(acc, E) / (double)m;
            yrep[N.yabs_off + r] = ldexp((double)aab, E) / (double)m;
        }
        return;
    }
    // open outputs: y(o) = (1/m) sum_j P(j) prod_sl S_sl[o_sl](j), each from the warp's
    // own stored spectra
    __threadfence_block();
    __syncwarp();
    for (int64_t o = 0; o < N.O; ++o) {
        int64_t oo[TNSK_MAX_OPEN_TENSORS] = {0, 0, 0, 0};
        for (int j = 0; j < N.n_open; ++j) {
            const OpenMode om = opens[N.open0 + j];
            const int64_t digit = (o / om.ostride) % om.dim;
#pragma unroll
            for (int sl = 0; sl < TNSK_MAX_OPEN_TENSORS; ++sl)
                if (sl == om.slot) oo[sl] += digit * om.tstride;
        }
        const C32* sp[TNSK_MAX_OPEN_TENSORS];
        int Eo = E;
#pragma unroll
        for (int sl = 0; sl < TNSK_MAX_OPEN_TENSORS; ++sl) {
            sp[sl] = nullptr;
            if (sl < N.n_ot) {
                const M1Tensor& Tt = tens[N.ot[sl]];
                sp[sl] = Sb + Tt.soff + oo[sl] * K;
                Eo += Eb[Tt.eoff + oo[sl]];
            }
        }
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < J; ++k) {
            const int q = k1L + J * k + J * J * cL;
            C32 v = P[k];
#pragma unroll
            for (int sl = 0; sl < TNSK_MAX_OPEN_TENSORS; ++sl)
                if (sl < N.n_ot) v = cmul(v, sp[sl][q]);
            acc += (q == 0 ? 1.0 : 2.0) * (double)v.x;
        }
        if (lane == 0) {
            float vM = PM;
#pragma unroll
            for (int sl = 0; sl < TNSK_MAX_OPEN_TENSORS; ++sl)
                if (sl < N.n_ot) vM *= sp[sl][M].x;
            acc += (double)vM;
        }
#pragma unroll
        for (int sft = 16; sft > 0; sft >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, sft);
        if (lane == 0) yr[o] = ldexp(acc, Eo) / (double)m;
    }
}

cudaError_t launch_m1_spectrum_warp(const M1Tensor* d_tens, const M1Net* d_nets, const OpenMode* d_opens,
                                    const int2* d_items, int n_items, const void* d_xs, const void* const* d_tws,
                                    void* d_spec, int* d_sexp, double* d_yrep, int log2m, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n_items + kWarps - 1) / kWarps);
    const float* xs = (const float*)d_xs;
    const C32* const* tws = (const C32* const*)d_tws;
    switch (log2m) {
        case 6: m1_spectrum_warp_kernel<0><<<blocks, kWarps * 32, 0, s>>>(d_tens, d_nets, d_opens, d_items, n_items, xs, tws, (C32*)d_spec, d_sexp, d_yrep); break;
        case 7: m1_spectrum_warp_kernel<1><<<blocks, kWarps * 32, 0, s>>>(d_tens, d_nets, d_opens, d_items, n_items, xs, tws, (C32*)d_spec, d_sexp, d_yrep); break;
        case 8: m1_spectrum_warp_kernel<2><<<blocks, kWarps * 32, 0, s>>>(d_tens, d_nets, d_opens, d_items, n_items, xs, tws, (C32*)d_spec, d_sexp, d_yrep); break;
        case 9: m1_spectrum_warp_kernel<3><<<blocks, kWarps * 32, 0, s>>>(d_tens, d_nets, d_opens, d_items, n_items, xs, tws, (C32*)d_spec, d_sexp, d_yrep); break;
        case 10: m1_spectrum_warp_kernel<4><<<blocks, kWarps * 32, 0, s>>>(d_tens, d_nets, d_opens, d_items, n_items, xs, tws, (C32*)d_spec, d_sexp, d_yrep); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace tnsk
