// m1_rowsort.cu -- row a2 (the method-1 sketch x_k = T_k vec(X_k), Eq. 1, hash form
// of Alg. 3) for large tensors streamed from HBM.
//
// The bin of entry (i, c) (i the leading mode's index, c the flat index of the other
// modes) is h_0(i) + h_J(c) mod m and its sign s_0(i) s_J(c), where h_J, s_J combine
// the other modes' count sketches. For a fixed column c and all rows i with the same
// bin h_0(i) = b, the entries land in the same bin b + h_J(c): their signed sum can be
// formed in a register and added once. So the rows are visited in the order of their
// leading-mode bins (a counting sort per tensor and rep, m1_rowsort_order_kernel), a
// lane owns one column (a warp reads 32 consecutive floats of a row: coalesced), adds
// s_0(i) X(i, c) into a register while the row bin stays the same, and adds the sum to
// the CTA's shared sketch when the bin changes. With n_0 rows over m bins that is
// about m (1 - e^{-n_0/m}) / n_0 shared atomics per entry (0.43 at n_0 = 2m) instead
// of one, and no per-entry hash arithmetic. Each repetition is a separate pass over
// the tensor (its rows sort differently), so the planner uses this form for tensors
// far larger than L2 and few repetitions per call.
#include <algorithm>

#include "kernels.cuh"
#include "plan.cuh"

namespace tnsk {

namespace {
constexpr int kRsThreads = 512;  // 16 warps: a strip of 512 columns
}

// Sorted rows of one (tensor, rep): packed words row << 15 | negative << 14 | bin, in
// the order of the bins. Counting sort in shared memory (m <= 2^14 counters).
__global__ void __launch_bounds__(1024) m1_rowsort_order_kernel(const M1Tensor* __restrict__ tens,
                                                                const M1Net* __restrict__ nets,
                                                                const M1RowSort* __restrict__ rs,
                                                                const uint32_t* __restrict__ tabs,
                                                                uint32_t* __restrict__ scratch) {
    extern __shared__ int32_t cnt[];  // [m]
    __shared__ int32_t warp_tot[32];
    const M1RowSort R = rs[blockIdx.x];
    const M1Tensor& T = tens[R.tensor];
    const M1Net& N = nets[R.net];
    const int m = (int)N.m;
    const uint32_t mask = (uint32_t)(m - 1);
    const int n0 = T.dims[0];
    const uint32_t* tab = tabs + N.tab_off + (int64_t)R.rep * N.L + T.tab[0];
    const bool comp = T.comp[0] != 0;
    auto word = [&](int i) {
        uint32_t w = tab[i];
        if (comp) w = (((uint32_t)m - (w & mask)) & mask) | (w & TNSK_SIGN_BIT);
        return w;
    };
    for (int b = threadIdx.x; b < m; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n0; i += blockDim.x) atomicAdd(&cnt[word(i) & mask], 1);
    __syncthreads();
    // exclusive prefix sum over the m counters: each thread scans a contiguous run
    const int per = (m + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(m, b0 + per);
    int run = 0;
    for (int b = b0; b < b1; ++b) run += cnt[b];
    // block-wide exclusive scan of the runs
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        int t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += v;
        }
        if (lane < nw) warp_tot[lane] = t;  // inclusive warp prefix
    }
    __syncthreads();
    int base = incl - run + (wid > 0 ? warp_tot[wid - 1] : 0);
    for (int b = b0; b < b1; ++b) {
        const int c = cnt[b];
        cnt[b] = base;
        base += c;
    }
    __syncthreads();
    uint32_t* out = scratch + R.order_off;
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        const uint32_t w = word(i);
        const int pos = atomicAdd(&cnt[w & mask], 1);
        out[pos] = ((uint32_t)i << 15) | ((w & TNSK_SIGN_BIT) ? (1u << 14) : 0u) | (w & mask);
    }
}

// One CTA slot: `count` consecutive (strip, sorted row) positions of the concatenation
// over the entries (see M1RowItem). The 16 warps of the CTA cover the 512 columns of one
// strip and walk the same rows, whose order words are staged in shared memory in
// chunks of kChunk; a lane's register sum is added to the shared sketch when the row
// bin changes and at the end of a chunk; the shared sketch goes to the entry's global
// sketch when the walk leaves the entry.
constexpr int kChunk = 512;

__global__ void __launch_bounds__(kRsThreads, 2) m1_rowsort_kernel(const M1Tensor* __restrict__ tens,
                                                                   const M1Net* __restrict__ nets,
                                                                   const M1RowSort* __restrict__ rs,
                                                                   const M1RowItem* __restrict__ items,
                                                                   const uint32_t* __restrict__ tabs,
                                                                   const uint32_t* __restrict__ scratch,
                                                                   float* __restrict__ xs) {
    extern __shared__ float x_sh[];  // [max m], then kChunk order words
    uint32_t* s_ord = nullptr;  // after the entry's m floats
    const M1RowItem it = items[blockIdx.x];
    int e = it.rs, strip = it.strip;
    int64_t k = it.k, left = it.count;
    while (left > 0) {
        // ---- entry e: its sketch in shared memory
        const M1RowSort R = rs[e];
        const M1Tensor& T = tens[R.tensor];
        const M1Net& N = nets[R.net];
        const int m = (int)N.m;
        const uint32_t mask = (uint32_t)(m - 1);
        const int64_t n0 = T.dims[0];
        const int64_t rl = T.numel / n0;
        const float* X = (const float*)T.data;
        const uint32_t* order = scratch + R.order_off;
        s_ord = reinterpret_cast<uint32_t*>(x_sh + m);
        __syncthreads();  // the previous entry's flush has read x_sh
        for (int b = threadIdx.x; b < m; b += blockDim.x) x_sh[b] = 0.f;
        while (left > 0) {
            // ---- strip `strip`: this lane's column and its combined word over modes
            // 1 .. order-1 (bins add; the sign bits' sum carries the sign product in bit 24)
            const int64_t c = (int64_t)strip * kRsThreads + threadIdx.x;
            const bool live = c < rl;
            uint32_t wc = 0;
            if (live) {
                const uint32_t* tab = tabs + N.tab_off + (int64_t)R.rep * N.L;
                int64_t rem = c;
                for (int d = T.order - 1; d >= 1; --d) {
                    const int64_t dim = T.dims[d];
                    const int64_t q = rem / dim;
                    const int x = (int)(rem - q * dim);
                    rem = q;
                    if (T.tab[d] < 0) continue;  // dim 1 (the planner admits no other open mode)
                    uint32_t w = tab[T.tab[d] + x];
                    if (T.comp[d]) w = (((uint32_t)m - (w & mask)) & mask) | (w & TNSK_SIGN_BIT);
                    wc += w;
                }
            }
            const uint32_t hc = wc & mask;
            const bool neg_c = (wc & TNSK_SIGN_BIT) != 0;
            const int64_t seg = min(left, n0 - k);  // rows of this strip in the slot
            for (int64_t k1 = k; k1 < k + seg; k1 += kChunk) {
                const int nk = (int)min((int64_t)kChunk, k + seg - k1);
                __syncthreads();  // the previous chunk's words are consumed
                for (int i = threadIdx.x; i < nk; i += blockDim.x) s_ord[i] = __ldg(order + k1 + i);
                __syncthreads();
                float z = 0.f;
                constexpr int kU = 16;  // rows per step: their loads in flight together
                for (int k0 = 0; k0 < nk; k0 += kU) {
                    uint32_t w[kU + 1];
                    float v[kU];
#pragma unroll
                    for (int u = 0; u <= kU; ++u) w[u] = k0 + u < nk ? s_ord[k0 + u] : 0u;
#pragma unroll
                    for (int u = 0; u < kU; ++u)
                        v[u] = (live && k0 + u < nk) ? __ldg(X + (int64_t)(w[u] >> 15) * rl + c) : 0.f;
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        if (k0 + u >= nk) break;
                        z += (w[u] & (1u << 14)) ? -v[u] : v[u];
                        // the next row's bin differs, or this is the chunk's last row
                        if (((w[u] ^ w[u + 1]) & mask) || k0 + u + 1 >= nk) {
                            if (live) atomicAdd(&x_sh[((w[u] & mask) + hc) & mask], neg_c ? -z : z);
                            z = 0.f;
                        }
                    }
                }
            }
            left -= seg;
            k = 0;
            if (++strip == R.strips) break;  // the entry is done
        }
        __syncthreads();
        float* gx = xs + N.x_off + (int64_t)R.rep * N.X + T.xoff;
        for (int b = threadIdx.x; b < m; b += blockDim.x) {
            const float val = x_sh[b];
            if (val != 0.f) atomicAdd(&gx[b], val);
        }
        ++e;
        strip = 0;
    }
}

int64_t m1_rowsort_slots() {
    static int64_t slots = 0;
    if (!slots) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
            cudaGetLastError();
            sms = 152;
        }
        slots = 2 * (int64_t)sms;  // two 512-thread CTAs per SM (launch bounds)
    }
    return slots;
}

cudaError_t launch_m1_rowsort(const BatchPlan& plan, unsigned char* base, float* xs, cudaStream_t s) {
    if (plan.m1.n_rs == 0) return cudaSuccess;
    const M1Tensor* tens = (const M1Tensor*)(base + plan.m1.tens_off);
    const M1Net* nets = (const M1Net*)(base + plan.m1.nets_off);
    const M1RowSort* rs = (const M1RowSort*)(base + plan.m1.rs_off);
    const M1RowItem* items = (const M1RowItem*)(base + plan.m1.rs_items_off);
    const uint32_t* tabs = (const uint32_t*)(base + plan.tabs_off);
    uint32_t* scratch = (uint32_t*)(base + plan.m1.rs_scratch_off);
    const size_t smem = (size_t)plan.m1.rs_max_m * 4;
    cudaFuncSetAttribute(m1_rowsort_order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    m1_rowsort_order_kernel<<<plan.m1.n_rs, 1024, smem, s>>>(tens, nets, rs, tabs, scratch);
    // the shared sketch, then one chunk of order words
    const size_t smem2 = smem + (size_t)kChunk * 4;
    cudaFuncSetAttribute(m1_rowsort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    m1_rowsort_kernel<<<plan.m1.n_rs_items, kRsThreads, smem2, s>>>(tens, nets, rs, items, tabs, scratch, xs);
    return cudaGetLastError();
}

}  // namespace tnsk
