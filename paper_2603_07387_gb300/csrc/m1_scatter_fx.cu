// m1_scatter_fx.cu -- row a2 (the method-1 sketch x_k = T_k vec(X_k), Eq. 1, by the
// hash form of the tensor sketch, Alg. 3) with the privatised bins accumulated in
// fixed point.
//
// FP32 shared-memory atomic adds to random bins run at about 0.95 T/s on GB300;
// 32-bit integer shared-memory adds whose result is unused run two to three times
// faster, while 64-bit or returning integer atomics do not. So every update is one
// 32-bit integer add of a quantised value, and exactness of the integer sums is kept
// by bounding them:
//   - a CTA processes its entries in batches of 16 entries per thread (8 above order
//     4), in groups of V consecutive entries (m1_fx_batch gives the batch size);
//   - per batch the CTA sums |x| over the batch (block reduction) and takes the
//     power of two 2^S with sum|x| 2^S <= 2^30; every entry becomes
//     q = round(x 2^S), so each bin's integer sum over the batch stays below 2^31 in
//     magnitude (any bin receives each entry at most once per rep), and the integer
//     adds are exact;
//   - after the batch the bins are converted back (q 2^-S, FP32) and added to an
//     FP32 accumulator in shared memory (items with more than one batch), or written
//     out directly (one batch).
// The only rounding beyond FP32's is the quantisation, |x 2^S - q| <= 1/2: an
// absolute error of at most 2^-31 sum|x| of the batch per entry.
// The loads of the next batch are issued before the current batch is scattered.
#include <type_traits>

#include "kernels.cuh"
#include "plan.cuh"

namespace tnsk {

namespace {

constexpr int kFxThreads = 512;

// 2^e as an FP32 value for -126 <= e <= 127 (exponent field only).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

}  // namespace

template <int MAXD, int V>
__global__ void __launch_bounds__(kFxThreads, 2) m1_scatter_fx_kernel(const M1Tensor* __restrict__ tens,
                                                                    const M1Net* __restrict__ nets,
                                                                    const M1Work* __restrict__ work,
                                                                    const uint32_t* __restrict__ tabs,
                                                                    float* __restrict__ xs) {
    // groups of V entries per thread and batch (fewer for high orders: registers)
    constexpr int U = (MAXD <= 4 ? 16 : 8) / V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ M1Tensor sT;
    __shared__ int32_t sbase[TNSK_MAX_ORDER], slo[TNSK_MAX_ORDER], scnt[TNSK_MAX_ORDER];
    __shared__ int32_t sTT;
    __shared__ float s_mass[3];
    // block-uniform per-slot data (slot s holds mode s - (MAXD - order): padding slots,
    // dim 1 and not contracted, come first, so the last mode is slot MAXD - 1), read from
    // shared memory where needed instead of held in every thread's registers
    __shared__ int32_t u_dim[MAXD], u_base[MAXD], u_lo[MAXD], u_step[MAXD], u_gofs[MAXD];
    __shared__ int64_t u_ostr[MAXD];
    __shared__ bool u_ctr[MAXD], u_comp[MAXD];
    const M1Work w = work[blockIdx.x];
    if (threadIdx.x == 0) {
        sT = tens[w.tensor];
        // per contracted mode: the staged index range [lo, lo + cnt) (mod dim); the whole
        // mode unless the work item's entries touch only part of it (w.ltab)
        int64_t P = 1;
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
        s_mass[0] = s_mass[1] = s_mass[2] = 0.f;
        int64_t sv = (int64_t)V * blockDim.x;  // the stride between a thread's groups
        for (int d = MAXD - 1; d >= 0; --d) {
            const int md = d - (MAXD - sT.order);
            const bool live = md >= 0;
            u_dim[d] = live ? (int32_t)sT.dims[md] : 1;
            u_base[d] = live ? sbase[md] : 0;
            u_lo[d] = live ? slo[md] : 0;
            u_ctr[d] = live && sT.tab[md] >= 0;
            u_comp[d] = u_ctr[d] && sT.comp[md];
            u_gofs[d] = u_ctr[d] ? sT.tab[md] : 0;
            u_ostr[d] = live ? sT.ostride[md] : 0;
            u_step[d] = (int32_t)(sv % u_dim[d]);
            sv /= u_dim[d];
        }
    }
    __syncthreads();
    const M1Net& N = nets[sT.net];
    const int64_t m = N.m;
    const uint32_t mask = (uint32_t)(m - 1);
    const int TT = sTT;
    const int nrep = w.nrep;
    const int order = sT.order;
    const int64_t O = sT.O;
    const int64_t nbins = (int64_t)nrep * O * m;
    const int64_t per_batch = (int64_t)V * U * blockDim.x;
    const int nbatch = (int)((w.end - w.begin + per_batch - 1) / per_batch);
    const bool multi = nbatch > 1;
    uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem_raw);
    const size_t tab_bytes = w.gtab ? 0 : (((size_t)nrep * TT * 4 + 15) & ~(size_t)15);
    int32_t* s_q = reinterpret_cast<int32_t*>(smem_raw + tab_bytes);  // [nrep][O][m] quantised sums
    float* s_acc = reinterpret_cast<float*>(s_q + nbins);               // [nrep][O][m] when multi

    // tables of this tensor's contracted modes for the batch of reps (complement applied)
    const int tab_words = w.gtab ? 0 : nrep * TT;
    for (int q = threadIdx.x; q < tab_words; q += blockDim.x) {
        const int r = q / TT;
        const int loc = q - r * TT;
        int d = 0;
        for (int dd = 0; dd < order; ++dd)
            if (sT.tab[dd] >= 0 && loc >= sbase[dd] && loc < sbase[dd] + scnt[dd]) d = dd;
        int i = slo[d] + (loc - sbase[d]);
        if (i >= sT.dims[d]) i -= (int)sT.dims[d];
        uint32_t word = tabs[N.tab_off + (int64_t)(w.rep0 + r) * N.L + sT.tab[d] + i];
        if (sT.comp[d]) word = (((uint32_t)m - (word & mask)) & mask) | (word & TNSK_SIGN_BIT);
        s_tab[q] = word;
    }
    for (int64_t q = threadIdx.x; q < nbins; q += blockDim.x) {
        s_q[q] = 0;
        if (multi) s_acc[q] = 0.f;
    }

    const int32_t* const dim = u_dim;
    const int32_t* const base = u_base;
    const int32_t* const lo = u_lo;
    const int32_t* const step = u_step;
    const int32_t* const gofs = u_gofs;
    const int64_t* const ostr = u_ostr;
    const bool* const ctr = u_ctr;
    const bool* const comp = u_comp;
    int dig[MAXD];  // this thread's multi-index (per slot)
    {
        int64_t f0 = w.begin + (int64_t)V * threadIdx.x;
#pragma unroll
        for (int d = MAXD - 1; d >= 0; --d) {
            dig[d] = (int)(f0 % dim[d]);
            f0 /= dim[d];
        }
    }
    const bool has_open = O > 1;
    const uint32_t* gt = tabs + N.tab_off + (int64_t)w.rep0 * N.L;
    const bool tab4 = V == 4 && !w.gtab && ctr[MAXD - 1] && (TT & 3) == 0 && (base[MAXD - 1] & 3) == 0 &&
                      (lo[MAXD - 1] & 3) == 0;
    __syncthreads();

    auto soff = [&](int d, int x) {
        const int r = x - lo[d];
        return base[d] + (r < 0 ? r + dim[d] : r);
    };
    // advance the multi-index by the stride (mixed-radix add with carries)
    auto advance = [&]() {
        int carry = 0;
#pragma unroll
        for (int d = MAXD - 1; d >= 0; --d) {
            const int t = dig[d] + step[d] + carry;
            carry = t >= dim[d];
            dig[d] = carry ? t - dim[d] : t;
        }
    };
    // Hoisted form: when the stride leaves every slot from d0 on unchanged (step digits
    // 0, so no carry reaches them), the last mode among them, and at most one contracted
    // slot dv below d0 changes, the words of the slots from d0 on are read once per rep
    // for all of a thread's groups (tensors whose trailing modes cover the stride, e.g.
    // the order-3 cores of tensor trains)
    int d0 = MAXD, dv = -1, nvar = 0;
#pragma unroll
    for (int d = MAXD - 1; d >= 0; --d)
        if (step[d] == 0 && d0 == d + 1) d0 = d;
#pragma unroll
    for (int d = 0; d < MAXD; ++d)
        if (d < d0 && ctr[d]) ++nvar, dv = d;
    const bool hoist = V == 4 && tab4 && d0 <= MAXD - 1 && !has_open && nvar <= 1;
    const int64_t fs = (int64_t)V * blockDim.x;  // stride between a thread's groups
    auto load = [&](float (&buf)[U][V], int64_t f) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t g = f + u * fs;
            if (V == 4) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (g < w.end) v = __ldg(reinterpret_cast<const float4*>((const float*)sT.data + g));
                buf[u][0] = v.x;
                buf[u][V > 1 ? 1 : 0] = v.y;
                buf[u][V > 2 ? 2 : 0] = v.z;
                buf[u][V > 3 ? 3 : 0] = v.w;
            } else {
                buf[u][0] = g < w.end ? load_as<float>(sT.data, sT.dtype, g) : 0.f;
            }
        }
    };

    float cur[U][V];
    int64_t f = w.begin + (int64_t)V * threadIdx.x;  // first entry of this thread's next group
    load(cur, f);
    int S = 0;
    for (int b = 0; b < nbatch; ++b) {
        // ---- the batch's mass sum |x| (block reduction) and its scale 2^S
        float part = 0.f;
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int j = 0; j < V; ++j) part += fabsf(cur[u][j]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        // three slots: slot (b + 1) % 3 was last read after barrier b - 2, and is next
        // written after barrier b
        if (threadIdx.x == 0) s_mass[(b + 1) % 3] = 0.f;
        if ((threadIdx.x & 31) == 0 && part > 0.f) atomicAdd(&s_mass[b % 3], part);
        __syncthreads();
        const float tot = s_mass[b % 3];
        if (tot > 0.f) {  // block-uniform; an all-zero batch adds nothing
            int ex;
            frexpf(tot, &ex);  // tot <= 2^ex
            S = 30 - ex;       // tot 2^S <= 2^30
            const int s1 = S / 2, s2 = S - S / 2;
            const float f1 = pow2f(s1), f2 = pow2f(s2);
            if (hoist) {
                // the slots from d0 on keep their digits across this thread's groups: their
                // words are read once per rep; one contracted slot dv below d0 varies
                int32_t qv[U][V];
                int ov[U];
                int64_t fg = f;
#pragma unroll
                for (int u = 0; u < U; ++u, fg += fs) {
#pragma unroll
                    for (int j = 0; j < V; ++j)
                        qv[u][j] = fg < w.end ? __float2int_rn((cur[u][j] * f1) * f2) : 0;
                    int od = 0;
#pragma unroll
                    for (int d = 0; d < MAXD; ++d)
                        if (d == dv) od = soff(d, dig[d]);
                    ov[u] = fg < w.end ? od : -1;
                    advance();
                }
                // word offsets of the fixed slots, -1 where a slot adds no word
                int hb[MAXD];
#pragma unroll
                for (int d = 0; d < MAXD; ++d)
                    hb[d] = (d == MAXD - 1 || (d >= d0 && ctr[d])) ? soff(d, dig[d]) : -1;  // unchanged by the advances
                auto rep_updates = [&](int r) {
                    const uint32_t* row = s_tab + r * TT;
                    uint32_t hc = 0;
#pragma unroll
                    for (int d = 0; d < MAXD - 1; ++d)
                        if (hb[d] >= 0) hc += row[hb[d]];
                    const uint4 wl = *reinterpret_cast<const uint4*>(row + hb[MAXD - 1]);
                    int32_t* qrow = s_q + (int64_t)r * m;
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (ov[u] < 0) continue;
                        const uint32_t h = hc + (dv >= 0 ? row[ov[u]] : 0u);
                        const uint32_t hw[4] = {h + wl.x, h + wl.y, h + wl.z, h + wl.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            atomicAdd(&qrow[hw[j] & mask], (hw[j] & TNSK_SIGN_BIT) ? -qv[u][j % V] : qv[u][j % V]);
                    }
                };
                int r = 0;
                for (; r + 1 < nrep; r += 2) {  // two reps at a time: twice the loads in flight
                    rep_updates(r);
                    rep_updates(r + 1);
                }
                if (r < nrep) rep_updates(r);
            } else {
                int64_t fg = f;
#pragma unroll
                for (int u = 0; u < U; ++u, fg += fs) {
                    if (fg < w.end) {
                        int32_t qv[V];
#pragma unroll
                        for (int j = 0; j < V; ++j) qv[j] = __float2int_rn((cur[u][j] * f1) * f2);
                        int64_t o = 0;
                        if (has_open)
#pragma unroll
                            for (int d = 0; d < MAXD; ++d) o += (int64_t)dig[d] * ostr[d];
                        int off[MAXD];  // staged word offsets (or global indices) of the group's digits
#pragma unroll
                        for (int d = 0; d < MAXD; ++d) off[d] = w.gtab ? gofs[d] + dig[d] : soff(d, dig[d]);
                        auto word_at = [&](int r, int d, int x) -> uint32_t {
                            if (w.gtab) {
                                uint32_t wd = __ldg(gt + (int64_t)r * N.L + x);
                                if (comp[d]) wd = (((uint32_t)m - (wd & mask)) & mask) | (wd & TNSK_SIGN_BIT);
                                return wd;
                            }
                            return s_tab[r * TT + x];
                        };
                        for (int r = 0; r < nrep; ++r) {
                            uint32_t h = 0;  // modes other than the last (V = 4) or all modes (V = 1)
#pragma unroll
                            for (int d = 0; d < MAXD; ++d)
                                if (ctr[d] && (V == 1 || d != MAXD - 1)) h += word_at(r, d, off[d]);
                            uint32_t wl[V];
                            if (V == 1) {
                                wl[0] = 0;
                            } else if (tab4) {
                                const uint4 t4 = *reinterpret_cast<const uint4*>(s_tab + r * TT + off[MAXD - 1]);
                                wl[0] = t4.x;
                                wl[V > 1 ? 1 : 0] = t4.y;
                                wl[V > 2 ? 2 : 0] = t4.z;
                                wl[V > 3 ? 3 : 0] = t4.w;
                            } else {
#pragma unroll
                                for (int j = 0; j < V; ++j)
                                    wl[j] = ctr[MAXD - 1] ? word_at(r, MAXD - 1, off[MAXD - 1] + j) : 0u;
                            }
                            int32_t* row = s_q + (int64_t)r * O * m;
#pragma unroll
                            for (int j = 0; j < V; ++j) {
                                const uint32_t hh = h + wl[j];
                                const int64_t oj = has_open ? o + (V > 1 ? j * ostr[MAXD - 1] : 0) : 0;
                                const int32_t q = (hh & TNSK_SIGN_BIT) ? -qv[j] : qv[j];
                                atomicAdd(&row[oj * m + (hh & mask)], q);
                            }
                        }
                    }
                    advance();
                }
            }
            if (multi && b + 1 < nbatch) {
                // fold this batch into the FP32 accumulator and clear the integer bins
                __syncthreads();
                const float g1 = pow2f(-s1), g2 = pow2f(-s2);
                for (int64_t q = threadIdx.x; q < nbins; q += blockDim.x) {
                    const int32_t v = s_q[q];
                    if (v != 0) {
                        s_acc[q] += ((float)v * g1) * g2;
                        s_q[q] = 0;
                    }
                }
            }
        } else {
            // an all-zero batch: skip its groups
#pragma unroll
            for (int u = 0; u < U; ++u) advance();
        }
        f += (int64_t)U * fs;
        if (b + 1 < nbatch) load(cur, f);
    }
    __syncthreads();
    // ---- out: the last batch's integer sums (scale 2^S) plus the accumulator
    const float g1 = pow2f(-(S / 2)), g2 = pow2f(-(S - S / 2));
    float* gx = xs + N.x_off + sT.xoff;
    const int per = (int)(O * m);
    for (int r = 0; r < nrep; ++r) {  // rep by rep: no division per bin
        float* gr = gx + (int64_t)(w.rep0 + r) * N.X;
        for (int ob = threadIdx.x; ob < per; ob += blockDim.x) {
            const int q = r * per + ob;
            float val = ((float)s_q[q] * g1) * g2;
            if (multi) val += s_acc[q];
            if (w.priv == 2)
                gr[ob] = val;  // this item owns these bins: no other CTA writes them
            else if (val != 0.f)
                atomicAdd(&gr[ob], val);
        }
    }
}

template <int MAXD>
static cudaError_t launch_fx_d(const M1Tensor* d_tens, const M1Net* d_nets, const M1Work* d_work, int n_work,
                               const uint32_t* d_tabs, float* d_xs, size_t smem, bool vec4, cudaStream_t s) {
    auto k = vec4 ? m1_scatter_fx_kernel<MAXD, 4> : m1_scatter_fx_kernel<MAXD, 1>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<n_work, kFxThreads, smem, s>>>(d_tens, d_nets, d_work, d_tabs, d_xs);
    return cudaGetLastError();
}

cudaError_t launch_m1_scatter_fx(const M1Tensor* d_tens, const M1Net* d_nets, const M1Work* d_work, int n_work,
                                 const uint32_t* d_tabs, float* d_xs, size_t smem, int max_order, bool vec4,
                                 cudaStream_t s) {
    if (n_work <= 0) return cudaSuccess;
    if (max_order <= 2) return launch_fx_d<2>(d_tens, d_nets, d_work, n_work, d_tabs, d_xs, smem, vec4, s);
    if (max_order <= 4) return launch_fx_d<4>(d_tens, d_nets, d_work, n_work, d_tabs, d_xs, smem, vec4, s);
    if (max_order <= 6) return launch_fx_d<6>(d_tens, d_nets, d_work, n_work, d_tabs, d_xs, smem, vec4, s);
    return launch_fx_d<TNSK_MAX_ORDER>(d_tens, d_nets, d_work, n_work, d_tabs, d_xs, smem, vec4, s);
}

int m1_fx_batch(int max_order, bool vec4) {
    const int per_thread = max_order <= 4 ? 16 : 8;
    (void)vec4;  // V entries x U groups = per_thread either way
    return per_thread * kFxThreads;
}

}  // namespace tnsk
