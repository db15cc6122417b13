// m1_scatter_fiber.cu -- row a2 (the method-1 sketch x_k = T_k vec(X_k), Eq. 1, by the
// hash form of the tensor sketch, Alg. 3) for FP32 tensors whose last mode is short
// (2 .. 16 indices) and whose entries cannot be read four at a time (the last dim is
// not a multiple of 4). A contracted last mode adds its word to each entry of a fiber;
// an open last mode instead sends the fiber's entries to consecutive output slots.
//
// The bin and sign of an entry are the sum of one table word per contracted mode
// (Alg. 3), so the strided walk of the fixed-point kernel reads q words per update
// (q = contracted modes). Here a thread takes whole fibers of the last mode instead:
// the words of the leading modes are summed once per fiber and rep, the last mode's L
// words once per rep for all of the thread's fibers, and every entry then costs one
// add and one shared-memory update: (q - 1) / L + 1 / UF table reads per update
// instead of q.
// Accumulation as in the fixed-point kernel (m1_scatter_fx.cu): per batch a block
// reduction of sum |x| gives 2^S with sum |x| 2^S <= 2^30, every entry becomes
// q = round(x 2^S), the 32-bit integer bin sums are exact, and after the batch the bins
// are folded into an FP32 accumulator (items of several batches) or written out; the
// only rounding beyond FP32's is the quantisation, at most 2^-31 sum|x| of the batch
// per entry.
#include "kernels.cuh"
#include "plan.cuh"

namespace tnsk {

namespace {

constexpr int kFibThreads = 512;
constexpr int kFibUF = 2;    // fibers per thread and batch
constexpr int kFibMaxL = 16;  // longest last mode taken

__device__ __forceinline__ float pow2f_fib(int e) { return __int_as_float((127 + e) << 23); }

}  // namespace

template <int MAXD>
__global__ void __launch_bounds__(kFibThreads, 1) m1_scatter_fiber_kernel(const M1Tensor* __restrict__ tens,
                                                                        const M1Net* __restrict__ nets,
                                                                        const M1Work* __restrict__ work,
                                                                        const uint32_t* __restrict__ tabs,
                                                                        float* __restrict__ xs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ M1Tensor sT;
    __shared__ int32_t sbase[TNSK_MAX_ORDER], slo[TNSK_MAX_ORDER], scnt[TNSK_MAX_ORDER];
    __shared__ int32_t sTT;
    __shared__ float s_mass[3];
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
    }
    __syncthreads();
    const M1Net& N = nets[sT.net];
    const int64_t m = N.m;
    const uint32_t mask = (uint32_t)(m - 1);
    const int TT = sTT;
    const int nrep = w.nrep;
    const int order = sT.order;
    const int L = sT.dims[order - 1];
    const int64_t O = sT.O;
    const int64_t nbins = (int64_t)nrep * O * m;
    const int64_t fib0 = w.begin / L, nfib = (w.end - w.begin) / L;
    const int64_t per_batch = (int64_t)kFibUF * blockDim.x;  // fibers
    const int nbatch = (int)((nfib + per_batch - 1) / per_batch);
    const bool multi = nbatch > 1;
    uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem_raw);
    const size_t tab_bytes = ((size_t)nrep * TT * 4 + 15) & ~(size_t)15;
    int32_t* s_q = reinterpret_cast<int32_t*>(smem_raw + tab_bytes);  // [nrep][O][m] quantised sums
    float* s_acc = reinterpret_cast<float*>(s_q + nbins);               // [nrep][O][m] when multi

    // tables of the contracted modes for the batch of reps (complement applied)
    for (int q = threadIdx.x; q < nrep * TT; q += blockDim.x) {
        const int r = q / TT;
        const int loc = q - r * TT;
        int d = 0;
        for (int dd = 0; dd < order; ++dd)
            if (sT.tab[dd] >= 0 && loc >= sbase[dd] && loc < sbase[dd] + scnt[dd]) d = dd;
        int i = slo[d] + (loc - sbase[d]);
        if (i >= sT.dims[d]) i -= sT.dims[d];
        uint32_t word = tabs[N.tab_off + (int64_t)(w.rep0 + r) * N.L + sT.tab[d] + i];
        if (sT.comp[d]) word = (((uint32_t)m - (word & mask)) & mask) | (word & TNSK_SIGN_BIT);
        s_tab[q] = word;
    }
    for (int64_t q = threadIdx.x; q < nbins; q += blockDim.x) {
        s_q[q] = 0;
        if (multi) s_acc[q] = 0.f;
    }
    // the last mode: contracted (its words, staged from index slo) or open (its stride)
    const bool last_ctr = sT.tab[order - 1] >= 0;
    // (an item holds whole fibers, so the last mode's staged range is the whole mode)
    const int lastb = sbase[order - 1];
    const int64_t lstep = last_ctr ? 0 : sT.ostride[order - 1] * m;
    __syncthreads();

    int S = 0;
    for (int b = 0; b < nbatch; ++b) {
        // ---- this batch's fibers of this thread: values, leading-mode word offsets, open offset
        float v[kFibUF][kFibMaxL];
        int po[kFibUF][MAXD > 1 ? MAXD - 1 : 1];
        int64_t oo[kFibUF];
        bool live[kFibUF];
        float part = 0.f;
#pragma unroll
        for (int u = 0; u < kFibUF; ++u) {
            const int64_t fl = (int64_t)b * per_batch + (int64_t)u * blockDim.x + threadIdx.x;  // fiber in item
            live[u] = fl < nfib;
            int64_t fg = fib0 + (live[u] ? fl : 0);
            const int64_t e0 = fg * L;
            oo[u] = 0;
            // digits of the leading modes, last of them fastest
#pragma unroll
            for (int d = MAXD - 2; d >= 0; --d) {
                po[u][d] = 0;
                if (d < order - 1) {
                    const int dim = sT.dims[d];
                    const int dig = (int)(fg % dim);
                    fg /= dim;
                    if (sT.tab[d] >= 0) {
                        const int rr = dig - slo[d];
                        po[u][d] = sbase[d] + (rr < 0 ? rr + dim : rr);
                    } else {
                        oo[u] += (int64_t)dig * sT.ostride[d];
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < kFibMaxL; ++i) {
                v[u][i] = (live[u] && i < L) ? load_as<float>(sT.data, sT.dtype, e0 + i) : 0.f;
                part += fabsf(v[u][i]);
            }
        }
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
            const float f1 = pow2f_fib(S / 2), f2 = pow2f_fib(S - S / 2);
            int32_t qv[kFibUF][kFibMaxL];
#pragma unroll
            for (int u = 0; u < kFibUF; ++u)
#pragma unroll
                for (int i = 0; i < kFibMaxL; ++i) qv[u][i] = __float2int_rn((v[u][i] * f1) * f2);
            for (int r = 0; r < nrep; ++r) {
                const uint32_t* row = s_tab + r * TT;
                uint32_t lw[kFibMaxL];  // the last mode's words, shared by the thread's fibers
#pragma unroll
                for (int i = 0; i < kFibMaxL; ++i) lw[i] = (last_ctr && i < L) ? row[lastb + i] : 0u;
                int32_t* qrow = s_q + (int64_t)r * O * m;
#pragma unroll
                for (int u = 0; u < kFibUF; ++u) {
                    if (!live[u]) continue;
                    uint32_t h = 0;
#pragma unroll
                    for (int d = 0; d < MAXD - 1; ++d)
                        if (d < order - 1 && sT.tab[d] >= 0) h += row[po[u][d]];
                    int32_t* orow = qrow + oo[u] * m;
#pragma unroll
                    for (int i = 0; i < kFibMaxL; ++i) {
                        if (i >= L) break;
                        const uint32_t hh = h + lw[i];
                        atomicAdd(&orow[i * lstep + (hh & mask)], (hh & TNSK_SIGN_BIT) ? -qv[u][i] : qv[u][i]);
                    }
                }
            }
            if (multi && b + 1 < nbatch) {
                // fold this batch into the FP32 accumulator and clear the integer bins
                __syncthreads();
                const float g1 = pow2f_fib(-(S / 2)), g2 = pow2f_fib(-(S - S / 2));
                for (int64_t q = threadIdx.x; q < nbins; q += blockDim.x) {
                    const int32_t val = s_q[q];
                    if (val != 0) {
                        s_acc[q] += ((float)val * g1) * g2;
                        s_q[q] = 0;
                    }
                }
            }
        }
        __syncthreads();
    }
    // ---- out: the last batch's integer sums (scale 2^S) plus the accumulator
    const float g1 = pow2f_fib(-(S / 2)), g2 = pow2f_fib(-(S - S / 2));
    float* gx = xs + N.x_off + sT.xoff;
    const int per = (int)(O * m);
    for (int q = threadIdx.x; q < (int)nbins; q += blockDim.x) {
        float val = ((float)s_q[q] * g1) * g2;
        if (multi) val += s_acc[q];
        const int r = q / per;
        const int ob = q - r * per;
        float* dst = &gx[(int64_t)(w.rep0 + r) * N.X + ob];
        if (w.priv == 2)
            *dst = val;  // this item owns these bins: no other CTA writes them
        else if (val != 0.f)
            atomicAdd(dst, val);
    }
}

template <int MAXD>
static cudaError_t launch_fiber_d(const M1Tensor* d_tens, const M1Net* d_nets, const M1Work* d_work, int n_work,
                                  const uint32_t* d_tabs, float* d_xs, size_t smem, cudaStream_t s) {
    auto k = m1_scatter_fiber_kernel<MAXD>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<n_work, kFibThreads, smem, s>>>(d_tens, d_nets, d_work, d_tabs, d_xs);
    return cudaGetLastError();
}

cudaError_t launch_m1_scatter_fiber(const M1Tensor* d_tens, const M1Net* d_nets, const M1Work* d_work, int n_work,
                                    const uint32_t* d_tabs, float* d_xs, size_t smem, int max_order,
                                    cudaStream_t s) {
    if (n_work <= 0) return cudaSuccess;
    if (max_order <= 2) return launch_fiber_d<2>(d_tens, d_nets, d_work, n_work, d_tabs, d_xs, smem, s);
    if (max_order <= 4) return launch_fiber_d<4>(d_tens, d_nets, d_work, n_work, d_tabs, d_xs, smem, s);
    if (max_order <= 6) return launch_fiber_d<6>(d_tens, d_nets, d_work, n_work, d_tabs, d_xs, smem, s);
    return launch_fiber_d<TNSK_MAX_ORDER>(d_tens, d_nets, d_work, n_work, d_tabs, d_xs, smem, s);
}

int64_t m1_fiber_batch(int L) { return (int64_t)kFibThreads * kFibUF * L; }

}  // namespace tnsk
