// method1.cu -- method 1 of the paper (Sec. 4.2, Eq. 1, Alg. 1): complement count
// sketches on every contraction, one tensor sketch per tensor, composition in
// the Fourier domain.
//
//   a2  m1_scatter_kernel   x_k[r] = T_k vec(X_k): signed scatter-add by the hash
//                           form of the tensor sketch (Alg. 3), shared-memory
//                           privatised bins for a batch of repetitions
//   a3  m1_spectrum_kernel  F x_k by a shared-memory real FFT
//   a4                      y_r = (1/m) sum_j prod_k (F x_k)(j) (Alg. 1 last line;
//                           open output entries per Corollary "full-to-partial-tc")
//   a9  combine_kernel      median of group means in FP64 (Theorem 1)
#include <algorithm>
#include <type_traits>

#include "fft.cuh"
#include "kernels.cuh"
#include "plan.cuh"

namespace tnsk {

// ---------------------------------------------------------------------------
// a2: scatter
// ---------------------------------------------------------------------------
// Shared memory: [nrep][TT] packed table words (complement applied), then the
// privatised bins [nrep][O][m] when w.priv. TT = sum of the contracted dims.
// Each thread walks entries f, f + S, f + 2S, ... (S = blockDim.x) keeping the
// multi-index of f in registers and adding the mixed-radix digits of S with
// carries, so no entry needs a division. MAXD bounds the tensor order.
// Tensors whose tables are large (w.gtab) read the table words from global memory
// instead (they stay in L2; within a warp the last mode's words are consecutive
// and the other modes' are shared), leaving shared memory to the bins.
// 512 threads: two CTAs (16 warps each) share an SM when the bins take ~96 KiB
constexpr int kScatterThreads = 512;

template <typename AccT, int MAXD>
__global__ void __launch_bounds__(kScatterThreads, 2) m1_scatter_kernel(const M1Tensor* __restrict__ tens,
                                                         const M1Net* __restrict__ nets,
                                                         const M1Work* __restrict__ work,
                                                         const uint32_t* __restrict__ tabs, AccT* __restrict__ xs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ M1Tensor sT;
    __shared__ int32_t sbase[TNSK_MAX_ORDER], slo[TNSK_MAX_ORDER], scnt[TNSK_MAX_ORDER];
    __shared__ int32_t sTT;
    const M1Work w = work[blockIdx.x];
    if (threadIdx.x == 0) {
        sT = tens[w.tensor];
        // per contracted mode: the staged index range [lo, lo + cnt) (mod dim); the whole
        // mode unless the work item's entries touch only part of it (w.ltab)
        int64_t P = 1;  // product of the dims after mode d
        for (int d = TNSK_MAX_ORDER - 1; d >= 0; --d) {
            slo[d] = 0;
            scnt[d] = d < sT.order ? (int32_t)sT.dims[d] : 0;
            if (d >= sT.order) continue;
            if (w.ltab && sT.dims[d] > 0) {
                const int64_t fb = w.begin / P, span = (w.end - 1) / P - fb + 1;
                if (span < sT.dims[d]) {
                    slo[d] = (int32_t)(fb % sT.dims[d]);
                    scnt[d] = (int32_t)span;
                }
            }
            P *= sT.dims[d];
        }
        int acc = 0;
        for (int d = 0; d < TNSK_MAX_ORDER; ++d) {
            sbase[d] = acc;
            if (d < sT.order && sT.tab[d] >= 0) acc += scnt[d];
        }
        sTT = acc;
    }
    __syncthreads();
    const M1Net& N = nets[sT.net];
    const int64_t m = N.m;
    const uint32_t mask = (uint32_t)(m - 1);
    const int TT = sTT;
    const int nrep = w.nrep;
    const int order = sT.order;
    uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem_raw);
    // bins after the staged tables (none in global-table mode): the plan sizes shared
    // memory the same way
    const size_t tab_bytes = w.gtab ? 0 : (((size_t)nrep * TT * 4 + 15) & ~(size_t)15);
    AccT* s_bin = reinterpret_cast<AccT*>(smem_raw + tab_bytes);

    // tables of this tensor's contracted modes for the batch of reps
    const int tab_words = w.gtab ? 0 : nrep * TT;  // fits shared memory
    for (int q = threadIdx.x; q < tab_words; q += blockDim.x) {
        int r = q / TT;
        int loc = q - r * TT;
        int d = 0;
        for (int dd = 0; dd < order; ++dd)
            if (sT.tab[dd] >= 0 && loc >= sbase[dd] && loc < sbase[dd] + scnt[dd]) d = dd;
        int i = slo[d] + (loc - sbase[d]);
        if (i >= sT.dims[d]) i -= (int)sT.dims[d];
        uint32_t word = tabs[N.tab_off + (int64_t)(w.rep0 + r) * N.L + sT.tab[d] + i];
        if (sT.comp[d]) word = (((uint32_t)m - (word & mask)) & mask) | (word & TNSK_SIGN_BIT);
        s_tab[q] = word;
    }
    const int64_t O = sT.O;
    const int64_t nbins = (int64_t)nrep * O * m;
    if (w.priv)
        for (int64_t q = threadIdx.x; q < nbins; q += blockDim.x) s_bin[q] = AccT(0);

    // block-uniform per-mode data in registers. Slot s holds mode s - (MAXD - order): the
    // padding slots (dim 1, not contracted) come first, so the last mode is slot MAXD - 1
    int dim[MAXD], base[MAXD], lo[MAXD], dig[MAXD], step[MAXD];
    bool ctr[MAXD];
    int64_t ostr[MAXD];
    const bool has_open = O > 1;
    // four entries per thread and step: FP32 data, 16-byte aligned, last dim a multiple
    // of 4 (so are the chunk bounds)
    const bool vec4 = sT.dtype == TNSK_F32 && order >= 1 && (sT.dims[order - 1] & 3) == 0 &&
                      ((uintptr_t)sT.data & 15) == 0 && (w.begin & 3) == 0 && (w.end & 3) == 0;
    {
        const int V = vec4 ? 4 : 1;
        int64_t f0 = w.begin + (int64_t)V * threadIdx.x;
        int64_t sv = (int64_t)V * blockDim.x;
#pragma unroll
        for (int d = MAXD - 1; d >= 0; --d) {
            const int md = d - (MAXD - order);  // the tensor mode in slot d
            const bool live = md >= 0;
            dim[d] = live ? sT.dims[md] : 1;
            base[d] = live ? sbase[md] : 0;
            lo[d] = live ? slo[md] : 0;
            ctr[d] = live && sT.tab[md] >= 0;
            ostr[d] = live ? sT.ostride[md] : 0;
            dig[d] = (int)(f0 % dim[d]);
            f0 /= dim[d];
            step[d] = (int)(sv % dim[d]);
            sv /= dim[d];
        }
    }
    __syncthreads();

    AccT* gx = xs + N.x_off + sT.xoff;  // + (rep0 + r) * N.X + o * m + b
    // global-table mode: mode d's words of rep r at gt + r * N.L + gofs[d] + index
    const uint32_t* gt = tabs + N.tab_off + (int64_t)w.rep0 * N.L;
    int32_t gofs[MAXD];
    bool gcomp[MAXD];
#pragma unroll
    for (int d = 0; d < MAXD; ++d) {
        const int md = d - (MAXD - order);
        gofs[d] = ctr[d] ? sT.tab[md] : 0;
        gcomp[d] = ctr[d] && sT.comp[md];
    }
    // staged rows of TT words with the last mode's words 16-byte aligned (it is contracted,
    // TT and its offset are multiples of 4; the vec4 path's index is one too)
    const bool tab4 = ctr[MAXD - 1] && (TT & 3) == 0 && (base[MAXD - 1] & 3) == 0 && (lo[MAXD - 1] & 3) == 0;
    // staged word offset of slot d's digit x (the staged range starts at lo, mod dim)
    auto soff = [&](int d, int x) {
        int r = x - lo[d];
        return base[d] + (r < 0 ? r + dim[d] : r);
    };
    // one table word of mode d at index off (rep r): staged or global, complement applied
    auto word_of = [&](auto global_tables, int r, int d, int off) -> uint32_t {
        if (decltype(global_tables)::value) {
            uint32_t wd = __ldg(gt + (int64_t)r * N.L + off);
            if (gcomp[d]) wd = (((uint32_t)m - (wd & mask)) & mask) | (wd & TNSK_SIGN_BIT);
            return wd;
        }
        return s_tab[r * TT + off];
    };
    auto add = [&](int r, int64_t o, uint32_t h, AccT v) {
        const AccT sv = (h & TNSK_SIGN_BIT) ? -v : v;
        const uint32_t b = h & mask;
        if (w.priv)
            atomicAdd(&s_bin[((int64_t)r * O + o) * m + b], sv);
        else
            atomicAdd(&gx[(int64_t)(w.rep0 + r) * N.X + o * m + b], sv);
    };
    // entries f = begin + V * (tid + k * blockDim.x) .. + V - 1: with V = 4 the four share
    // every digit but the last (the last mode's dim is a multiple of 4), come in one
    // 16-byte load, and share the other modes' table words
    auto entries = [&](auto global_tables, auto vec) {
        constexpr bool kG = decltype(global_tables)::value;
        constexpr int V = decltype(vec)::value;
        constexpr int L = MAXD - 1;  // the tensor's last mode
        // the next step's entries are loaded before this step's adds (one load in flight
        // per thread while it works, which matters when the tensor streams from HBM)
        const int64_t fs = (int64_t)V * blockDim.x;
        int64_t f = w.begin + (int64_t)V * threadIdx.x;
        float4 qn = make_float4(0.f, 0.f, 0.f, 0.f);
        AccT vn = AccT(0);
        if (f < w.end) {
            if (V == 4)
                qn = __ldg(reinterpret_cast<const float4*>((const float*)sT.data + f));
            else
                vn = load_as<AccT>(sT.data, sT.dtype, f);
        }
        for (; f < w.end; f += fs) {
            AccT v[V];
            if (V == 4) {
                v[0] = (AccT)qn.x;
                v[V > 1 ? 1 : 0] = (AccT)qn.y;
                v[V > 2 ? 2 : 0] = (AccT)qn.z;
                v[V > 3 ? 3 : 0] = (AccT)qn.w;
            } else {
                v[0] = vn;
            }
            if (f + fs < w.end) {
                if (V == 4)
                    qn = __ldg(reinterpret_cast<const float4*>((const float*)sT.data + f + fs));
                else
                    vn = load_as<AccT>(sT.data, sT.dtype, f + fs);
            }
            int off[MAXD];
            int64_t o = 0;
#pragma unroll
            for (int d = 0; d < MAXD; ++d) {
                off[d] = kG ? gofs[d] + dig[d] : soff(d, dig[d]);
                if (has_open) o += (int64_t)dig[d] * ostr[d];
            }
            for (int r = 0; r < nrep; ++r) {
                uint32_t h = 0;  // the modes other than the last (V = 4) or all modes (V = 1)
#pragma unroll
                for (int d = 0; d < MAXD; ++d)
                    if (ctr[d] && (V == 1 || d != L)) h += word_of(global_tables, r, d, off[d]);
                if (V == 1) {
                    add(r, o, h, v[0]);
                } else {
                    // the last mode's four words: one 16-byte load when the staged row allows
                    uint32_t wl[V];
                    if (!kG && tab4) {
                        const uint4 q = *reinterpret_cast<const uint4*>(s_tab + r * TT + off[L]);
                        wl[0] = q.x;
                        wl[V > 1 ? 1 : 0] = q.y;
                        wl[V > 2 ? 2 : 0] = q.z;
                        wl[V > 3 ? 3 : 0] = q.w;
                    } else {
#pragma unroll
                        for (int j = 0; j < V; ++j) wl[j] = ctr[L] ? word_of(global_tables, r, L, off[L] + j) : 0u;
                    }
#pragma unroll
                    for (int j = 0; j < V; ++j) add(r, has_open ? o + j * ostr[L] : o, h + wl[j], v[j]);
                }
            }
            // advance the multi-index by V * blockDim.x (mixed-radix add with carries)
            int carry = 0;
#pragma unroll
            for (int d = MAXD - 1; d >= 0; --d) {
                int t = dig[d] + step[d] + carry;
                carry = t >= dim[d];
                dig[d] = carry ? t - dim[d] : t;
            }
        }
    };
    // Hoisted form of the staged vec4 path: when the stride of a thread's entries leaves
    // every slot from d0 on unchanged (their step digits are 0, so no carry reaches them),
    // the last mode among them, and exactly one contracted slot dv below d0 changes, a
    // thread takes up to 4 of its entries at once and, per rep, reads the unchanged
    // slots' words once (the last mode's four as one 16-byte load) and one word of dv
    // per entry, instead of every word per entry.
    int d0 = MAXD, dv = -1, nvar = 0;
#pragma unroll
    for (int d = MAXD - 1; d >= 0; --d)
        if (step[d] == 0 && d0 == d + 1) d0 = d;
#pragma unroll
    for (int d = 0; d < MAXD; ++d)
        if (d < d0 && ctr[d]) ++nvar, dv = d;
    const bool hoist = vec4 && !w.gtab && tab4 && d0 <= MAXD - 1 && !has_open && nvar == 1;
    auto entries_hoisted = [&]() {
        constexpr int L = MAXD - 1;
        constexpr int KG = 4;
        const int64_t S = 4 * (int64_t)blockDim.x;
        int hb[MAXD];  // offsets of the unchanged slots' words
#pragma unroll
        for (int d = 0; d < MAXD; ++d) hb[d] = soff(d, dig[d]);
        int64_t f = w.begin + 4 * (int64_t)threadIdx.x;
        while (f < w.end) {
            float4 q[KG];
            int ov[KG];
            int kn = 0;
#pragma unroll
            for (int k = 0; k < KG; ++k) {
                q[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                ov[k] = 0;
                if (f < w.end) {
                    q[k] = __ldg(reinterpret_cast<const float4*>((const float*)sT.data + f));
                    int od = 0;
#pragma unroll
                    for (int d = 0; d < MAXD; ++d)
                        if (d == dv) od = soff(d, dig[d]);
                    ov[k] = od;
                    ++kn;
                    f += S;
                    int carry = 0;  // advance the changing slots (below d0) by the stride
#pragma unroll
                    for (int d = MAXD - 1; d >= 0; --d) {
                        if (d >= d0) continue;
                        const int t = dig[d] + step[d] + carry;
                        carry = t >= dim[d];
                        dig[d] = carry ? t - dim[d] : t;
                    }
                }
            }
            for (int r = 0; r < nrep; ++r) {
                const uint32_t* row = s_tab + r * TT;
                uint32_t hc = 0;
#pragma unroll
                for (int d = 0; d < L; ++d)
                    if (d >= d0 && ctr[d]) hc += row[hb[d]];
                const uint4 wl = *reinterpret_cast<const uint4*>(row + hb[L]);
#pragma unroll
                for (int k = 0; k < KG; ++k) {
                    if (k >= kn) break;
                    const uint32_t h = hc + row[ov[k]];
                    add(r, 0, h + wl.x, (AccT)q[k].x);
                    add(r, 0, h + wl.y, (AccT)q[k].y);
                    add(r, 0, h + wl.z, (AccT)q[k].z);
                    add(r, 0, h + wl.w, (AccT)q[k].w);
                }
            }
        }
    };
    if (vec4) {
        if (w.gtab)
            entries(std::true_type{}, std::integral_constant<int, 4>{});
        else if (hoist && sizeof(AccT) == 4)
            entries_hoisted();
        else
            entries(std::false_type{}, std::integral_constant<int, 4>{});
    } else {
        if (w.gtab)
            entries(std::true_type{}, std::integral_constant<int, 1>{});
        else
            entries(std::false_type{}, std::integral_constant<int, 1>{});
    }
    if (!w.priv) return;
    __syncthreads();
    // the bins of reps [rep0, rep0 + nrep) of this tensor are contiguous per rep
    const int per = (int)(O * m);  // the bins fit shared memory
    for (int q = threadIdx.x; q < (int)nbins; q += blockDim.x) {
        AccT val = s_bin[q];
        int r = q / per;
        int ob = q - r * per;
        AccT* dst = &gx[(int64_t)(w.rep0 + r) * N.X + ob];
        if (w.priv == 2)
            *dst = val;  // this item owns these bins: no other CTA writes them
        else if (val != AccT(0))
            atomicAdd(dst, val);
    }
}

// ---------------------------------------------------------------------------
// a3 + a4: spectra, Hadamard product, bin sum
// ---------------------------------------------------------------------------
// One CTA per (network, rep). The sketches of the network (one per tensor, or
// one per open index of a tensor with open legs) are transformed G at a time:
// shared memory holds z [G][M] (packed complex sketches, FFT in place) and
// P [M+1] (running Hadamard product of the folded spectra, scaled by 2^-E).
template <typename T>
__global__ void __launch_bounds__(256) m1_spectrum_kernel(const M1Tensor* __restrict__ tens,
                                                          const M1Net* __restrict__ nets,
                                                          const OpenMode* __restrict__ opens,
                                                          const int2* __restrict__ items, const T* __restrict__ xs,
                                                          const Cplx<T>* const* __restrict__ tws,
                                                          Cplx<T>* __restrict__ spec, int* __restrict__ sexp,
                                                          double* __restrict__ yrep, int gmax) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int kMaxG = 16;
    __shared__ int s_k[kMaxG];       // tensor of each sketch in the group
    __shared__ int64_t s_o[kMaxG];   // its open index
    __shared__ int64_t s_x[kMaxG];   // offset of its sketch in the rep's sketch vector
    __shared__ int64_t s_so[kMaxG];  // its open-spectrum offset, -1 when folded into P
    __shared__ int64_t s_eo[kMaxG];  // its exponent slot
    __shared__ unsigned long long s_max[kMaxG];  // bits of max |Re|,|Im| as a double (non-negative: ordered)
    __shared__ int s_e[kMaxG];      // its power-of-two exponent
    __shared__ double dred[32];
    const int2 it = items[blockIdx.x];
    const M1Net& N = nets[it.x];
    const int r = it.y;
    const int64_t m = N.m;
    const int log2m = N.log2m;
    const int log2M = log2m > 0 ? log2m - 1 : 0;
    const int M = 1 << log2M;
    const int K = m == 1 ? 1 : M + 1;
    Cplx<T>* z = reinterpret_cast<Cplx<T>*>(smem_raw);
    Cplx<T>* P = z + (size_t)gmax * M;
    Cplx<T>* tw = P + M + 1;  // twiddles of this m, copied once
    const int64_t O = N.O;
    if (O == 0) return;
    for (int k = threadIdx.x; k < K; k += blockDim.x) P[k] = {T(1), T(0)};
    {
        const Cplx<T>* twg = tws[log2m];
        for (int k = threadIdx.x; k < M; k += blockDim.x) tw[k] = twg[k];
    }
    int E = 0;  // P holds 2^-E prod_k F x_k
    const T* xr = xs + N.x_off + (int64_t)r * N.X;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int k_cur = 0;
    int64_t o_cur = 0;
    while (k_cur < N.p) {
        // ---- the next group of up to gmax sketches (same walk in every thread)
        int G = 0;
        while (G < gmax && k_cur < N.p) {
            const M1Tensor& Tk = tens[N.t0 + k_cur];
            const int64_t nsk = Tk.soff < 0 ? 1 : Tk.O;
            if (threadIdx.x == 0) {
                s_k[G] = k_cur;
                s_o[G] = o_cur;
                s_x[G] = Tk.xoff + o_cur * m;
                s_so[G] = Tk.soff < 0 ? -1 : Tk.soff + o_cur * K;
                s_eo[G] = Tk.soff < 0 ? -1 : Tk.eoff + o_cur;
                s_max[G] = 0;
            }
            ++G;
            if (++o_cur >= nsk) {
                o_cur = 0;
                ++k_cur;
            }
        }
        __syncthreads();
        // ---- load as packed complex z[n] = x[2n] + i x[2n+1] (z[0] = x[0] when m = 1)
        for (int idx = threadIdx.x; idx < G * M; idx += blockDim.x) {
            const int g = idx >> log2M, n = idx & (M - 1);
            const T* x = xr + s_x[g];
            z[idx] = m == 1 ? Cplx<T>{x[0], T(0)} : Cplx<T>{x[2 * n], x[2 * n + 1]};
        }
        __syncthreads();
        if (m > 1) block_fft_dif(z, G, log2M, tw);
        // ---- per-sketch magnitude for the power-of-two scaling
        for (int g = 0; g < G; ++g) {
            T mx = T(0);
            for (int kk = threadIdx.x; kk < K; kk += blockDim.x) {
                Cplx<T> X = m == 1 ? z[g * M] : unpack_bin(z + g * M, kk, log2M, tw);
                mx = fmax(mx, fmax(fabs(X.x), fabs(X.y)));
            }
#pragma unroll
            for (int sft = 16; sft > 0; sft >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, sft));
            if (lane == 0 && mx > T(0)) atomicMax(&s_max[g], (unsigned long long)__double_as_longlong((double)mx));
        }
        __syncthreads();
        if (threadIdx.x < G) {
            int e = 0;
            const double mx = __longlong_as_double((long long)s_max[threadIdx.x]);
            if (mx > 0.0) frexp(mx, &e);
            s_e[threadIdx.x] = e;  // 2^-e F x has entries below 1 in magnitude
        }
        __syncthreads();
        // ---- fold into P (tensors without open legs) or keep the open spectra
        for (int kk = threadIdx.x; kk < K; kk += blockDim.x) {
            Cplx<T> pk = P[kk];
            for (int g = 0; g < G; ++g) {
                Cplx<T> X = m == 1 ? z[g * M] : unpack_bin(z + g * M, kk, log2M, tw);
                const T sc = (T)ldexp(1.0, -s_e[g]);
                X.x *= sc;
                X.y *= sc;
                if (s_so[g] < 0)
                    pk = cmul(pk, X);
                else
                    spec[N.spec_off + (int64_t)r * N.spec_per_rep + s_so[g] + kk] = X;
            }
            P[kk] = pk;
        }
        for (int g = 0; g < G; ++g) {
            if (s_so[g] < 0)
                E += s_e[g];
            else if (threadIdx.x == 0)
                sexp[N.exp_off + (int64_t)r * N.exp_per_rep + s_eo[g]] = s_e[g];
        }
        __syncthreads();
    }
    // y_r(o) = (1/m) sum_j prod_k (F x_k[o_k])(j); the full spectrum is Hermitian,
    // so sum_j = P[0] + P[M] + 2 Re sum_{0<k<M} P[k] (m >= 2).
    double* yr = yrep + N.y_off + (int64_t)r * O;
    if (N.n_ot == 0) {
        double acc = 0;  // the sum, and the magnitude sum as sum (|Re| + |Im|) (FP64 criterion)
        T aab = T(0);
        for (int k = threadIdx.x; k < K; k += blockDim.x) {
            double wgt = (m == 1 || k == 0 || k == M) ? 1.0 : 2.0;
            acc += wgt * (double)P[k].x;
            aab += T(wgt) * (fabs(P[k].x) + fabs(P[k].y));
        }
#pragma unroll
        for (int sft = 16; sft > 0; sft >>= 1) {
            acc += __shfl_xor_sync(0xffffffffu, acc, sft);
            aab += __shfl_xor_sync(0xffffffffu, aab, sft);
        }
        if (lane == 0) {
            dred[warp] = acc;
            dred[16 + warp] = (double)aab;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0, ta = 0;
            for (int q = 0; q < nw; ++q) {
                t += dred[q];
                ta += dred[16 + q];
            }
            yr[0] = ldexp(t, E) / (double)m;
            yrep[N.yabs_off + r] = ldexp(ta, E) / (double)m;
        }
        return;
    }
    // open outputs: one warp per output entry
    const Cplx<T>* Sb = spec + N.spec_off + (int64_t)r * N.spec_per_rep;
    const int* Eb = sexp + N.exp_off + (int64_t)r * N.exp_per_rep;
    for (int64_t o = warp; o < O; o += nw) {
        int64_t oo[TNSK_MAX_OPEN_TENSORS] = {0, 0, 0, 0};
        for (int j = 0; j < N.n_open; ++j) {
            const OpenMode om = opens[N.open0 + j];
            int64_t digit = (o / om.ostride) % om.dim;
#pragma unroll
            for (int sl = 0; sl < TNSK_MAX_OPEN_TENSORS; ++sl)
                if (sl == om.slot) oo[sl] += digit * om.tstride;
        }
        const Cplx<T>* sp[TNSK_MAX_OPEN_TENSORS];
        int Eo = E;
#pragma unroll
        for (int sl = 0; sl < TNSK_MAX_OPEN_TENSORS; ++sl) {
            if (sl < N.n_ot) {
                const M1Tensor& Tt = tens[N.ot[sl]];
                sp[sl] = Sb + Tt.soff + oo[sl] * K;
                Eo += Eb[Tt.eoff + oo[sl]];
            } else {
                sp[sl] = nullptr;
            }
        }
        double acc = 0;
        for (int k = lane; k < K; k += 32) {
            Cplx<T> v = P[k];
#pragma unroll
            for (int sl = 0; sl < TNSK_MAX_OPEN_TENSORS; ++sl)
                if (sl < N.n_ot) v = cmul(v, sp[sl][k]);
            double wgt = (m == 1 || k == 0 || k == M) ? 1.0 : 2.0;
            acc += wgt * (double)v.x;
        }
#pragma unroll
        for (int sft = 16; sft > 0; sft >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, sft);
        if (lane == 0) yr[o] = ldexp(acc, Eo) / (double)m;
    }
}

// ---------------------------------------------------------------------------
// a9: median of group means (Theorem 1), FP64
// ---------------------------------------------------------------------------
__global__ void combine_kernel(const CombineItem* __restrict__ items, int n_items, const double* __restrict__ yrep) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_items; i += gridDim.x * blockDim.x) {
        const CombineItem c = items[i];
        const double* y = yrep + c.y_off;
        const int gs = c.R / c.groups;
        double med[64];
        for (int g = 0; g < c.groups; ++g) {
            double s = 0;
            for (int r = g * gs; r < (g + 1) * gs; ++r) s += y[(int64_t)r * c.O + c.o];
            double mean = s / gs;
            int q = g;  // insertion sort
            while (q > 0 && med[q - 1] > mean) {
                med[q] = med[q - 1];
                --q;
            }
            med[q] = mean;
        }
        const int g = c.groups;
        c.out[c.o] = (g & 1) ? med[g / 2] : 0.5 * (med[g / 2 - 1] + med[g / 2]);
        if (c.per_rep)
            for (int r = 0; r < c.R; ++r) c.per_rep[(int64_t)r * c.ps + c.o] = y[(int64_t)r * c.O + c.o];
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename AccT, int MAXD>
cudaError_t launch_scatter_d(const M1Tensor* d_tens, const M1Net* d_nets, const M1Work* d_work, int n_work,
                             const uint32_t* d_tabs, AccT* d_xs, size_t smem, cudaStream_t s) {
    auto k = m1_scatter_kernel<AccT, MAXD>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<n_work, kScatterThreads, smem, s>>>(d_tens, d_nets, d_work, d_tabs, d_xs);
    return cudaGetLastError();
}

template <typename AccT>
cudaError_t launch_m1_scatter_t(const M1Tensor* d_tens, const M1Net* d_nets, const M1Work* d_work, int n_work,
                                const uint32_t* d_tabs, AccT* d_xs, size_t smem, int max_order, cudaStream_t s) {
    if (n_work <= 0) return cudaSuccess;
    if (max_order <= 2) return launch_scatter_d<AccT, 2>(d_tens, d_nets, d_work, n_work, d_tabs, d_xs, smem, s);
    if (max_order <= 4) return launch_scatter_d<AccT, 4>(d_tens, d_nets, d_work, n_work, d_tabs, d_xs, smem, s);
    if (max_order <= 6) return launch_scatter_d<AccT, 6>(d_tens, d_nets, d_work, n_work, d_tabs, d_xs, smem, s);
    return launch_scatter_d<AccT, TNSK_MAX_ORDER>(d_tens, d_nets, d_work, n_work, d_tabs, d_xs, smem, s);
}

cudaError_t launch_m1_scatter(const M1Tensor* d_tens, const M1Net* d_nets, const M1Work* d_work, int n_work,
                              const uint32_t* d_tabs, void* d_xs, bool fp64, size_t smem, int max_order,
                              cudaStream_t s) {
    if (fp64)
        return launch_m1_scatter_t<double>(d_tens, d_nets, d_work, n_work, d_tabs, (double*)d_xs, smem, max_order, s);
    return launch_m1_scatter_t<float>(d_tens, d_nets, d_work, n_work, d_tabs, (float*)d_xs, smem, max_order, s);
}

cudaError_t launch_m1_spectrum(const M1Tensor* d_tens, const M1Net* d_nets, const OpenMode* d_opens,
                               const int2* d_items, int n_items, const void* d_xs, const void* const* d_tws,
                               void* d_spec, int* d_sexp, double* d_yrep, bool fp64, int max_log2m,
                               cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    const int M = max_log2m > 0 ? 1 << (max_log2m - 1) : 1;
    // sketches per FFT pass: up to 32 KiB of them, at most 8 (occupancy over batching)
    const size_t csz = fp64 ? sizeof(Cplx<double>) : sizeof(Cplx<float>);
    int gmax = (int)std::max<size_t>(1, std::min<size_t>(8, (32 * 1024) / (M * csz)));
    size_t smem = ((size_t)gmax * M + M + 1 + M) * csz;
    if (fp64) {
        auto k = m1_spectrum_kernel<double>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<n_items, 256, smem, s>>>(d_tens, d_nets, d_opens, d_items, (const double*)d_xs,
                                     (const Cplx<double>* const*)d_tws, (Cplx<double>*)d_spec, d_sexp, d_yrep, gmax);
    } else {
        auto k = m1_spectrum_kernel<float>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<n_items, 256, smem, s>>>(d_tens, d_nets, d_opens, d_items, (const float*)d_xs,
                                     (const Cplx<float>* const*)d_tws, (Cplx<float>*)d_spec, d_sexp, d_yrep, gmax);
    }
    return cudaGetLastError();
}

cudaError_t launch_m1_scatter_list(const BatchPlan& plan, unsigned char* base, void* xs, bool fp64, int list,
                                   cudaStream_t s) {
    static const int kClassOrder[M1Plan::kOrderClasses] = {2, 4, 6, TNSK_MAX_ORDER};
    const M1Tensor* tens = (const M1Tensor*)(base + plan.m1.tens_off);
    const M1Net* nets = (const M1Net*)(base + plan.m1.nets_off);
    const M1Work* work = (const M1Work*)(base + plan.m1.work_off);
    const uint32_t* tabs = (const uint32_t*)(base + plan.tabs_off);
    const int c = list % M1Plan::kOrderClasses, k = list / M1Plan::kOrderClasses;
    if (k == 0)
        return launch_m1_scatter(tens, nets, work + plan.m1.work_first[list], plan.m1.work_count[list], tabs, xs, fp64,
                                 plan.m1.class_smem[list], kClassOrder[c], s);
    if (fp64) return cudaSuccess;
    if (k == 3)
        return launch_m1_scatter_fiber(tens, nets, work + plan.m1.work_first[list], plan.m1.work_count[list], tabs,
                                       (float*)xs, plan.m1.class_smem[list], kClassOrder[c], s);
    return launch_m1_scatter_fx(tens, nets, work + plan.m1.work_first[list], plan.m1.work_count[list], tabs,
                                (float*)xs, plan.m1.class_smem[list], kClassOrder[c], k == 1, s);
}

cudaError_t launch_m1_scatters(const BatchPlan& plan, unsigned char* base, void* xs, bool fp64, cudaStream_t s) {
    const M1Tensor* tens = (const M1Tensor*)(base + plan.m1.tens_off);
    const M1Net* nets = (const M1Net*)(base + plan.m1.nets_off);
    const M1Work* work = (const M1Work*)(base + plan.m1.work_off);
    const uint32_t* tabs = (const uint32_t*)(base + plan.tabs_off);
    static const int kClassOrder[M1Plan::kOrderClasses] = {2, 4, 6, TNSK_MAX_ORDER};
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < M1Plan::kOrderClasses && e == cudaSuccess; ++c)
        e = launch_m1_scatter(tens, nets, work + plan.m1.work_first[c], plan.m1.work_count[c], tabs, xs, fp64,
                              plan.m1.class_smem[c], kClassOrder[c], s);
    // FP32 privatised items: the fixed-point kernel (four-entry loads, then one-entry),
    // then the fiber kernel
    for (int k = 1; k <= 3 && !fp64; ++k)
        for (int c = 0; c < M1Plan::kOrderClasses && e == cudaSuccess; ++c) {
            const int l = c + M1Plan::kOrderClasses * k;
            e = k == 3 ? launch_m1_scatter_fiber(tens, nets, work + plan.m1.work_first[l], plan.m1.work_count[l], tabs,
                                                 (float*)xs, plan.m1.class_smem[l], kClassOrder[c], s)
                       : launch_m1_scatter_fx(tens, nets, work + plan.m1.work_first[l], plan.m1.work_count[l], tabs,
                                              (float*)xs, plan.m1.class_smem[l], kClassOrder[c], k == 1, s);
        }
    // large FP32 tensors streamed from HBM: the row-sorted form
    if (e == cudaSuccess && !fp64) e = launch_m1_rowsort(plan, base, (float*)xs, s);
    return e;
}

cudaError_t launch_m1_spectra(const BatchPlan& plan, unsigned char* base, const void* xs, const void* const* tws,
                              bool fp64, cudaStream_t s) {
    const M1Tensor* tens = (const M1Tensor*)(base + plan.m1.tens_off);
    const M1Net* nets = (const M1Net*)(base + plan.m1.nets_off);
    const int2* items = (const int2*)(base + plan.m1.items_off);
    double* yrep = (double*)(base + plan.yrep_off);
    cudaError_t e = launch_m1_spectrum(tens, nets, (const OpenMode*)(base + plan.m1.opens_off), items,
                                       plan.m1.n_items, xs, tws, base + plan.m1.spec_off,
                                       (int*)(base + plan.m1.sexp_off), yrep, fp64, plan.m1.max_log2m, s);
    for (int sl = 0; sl < M1Plan::kWarpSlots && e == cudaSuccess; ++sl)
        e = launch_m1_spectrum_warp(tens, nets, (const OpenMode*)(base + plan.m1.opens_off),
                                    items + plan.m1.warp_first[sl], plan.m1.warp_count[sl], xs, tws,
                                    base + plan.m1.spec_off, (int*)(base + plan.m1.sexp_off), yrep, 6 + sl, s);
    if (e == cudaSuccess)
        e = launch_m1_mid(tens, nets, (const int4*)(base + plan.m1.mfft_off), plan.m1.n_mfft,
                          (const int4*)(base + plan.m1.mprod_off), plan.m1.n_mprod, plan.m1.mid_max_log2m, xs, tws,
                          base + plan.m1.lspec_off, yrep, fp64, s);
    if (e == cudaSuccess)
        e = launch_m1_large(tens, nets, (const int4*)(base + plan.m1.lfft_off), plan.m1.n_lfft,
                            (const int4*)(base + plan.m1.lprod_off), plan.m1.n_lprod, plan.m1.lrows_smem, xs, tws,
                            base + plan.m1.lspec_off, yrep, fp64, s);
    return e;
}

cudaError_t launch_combine(const CombineItem* d_items, int n_items, const double* d_yrep, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    int blocks = (n_items + 127) / 128;
    if (blocks > 152 * 16) blocks = 152 * 16;
    combine_kernel<<<blocks, 128, 0, s>>>(d_items, n_items, d_yrep);
    return cudaGetLastError();
}

}  // namespace tnsk
