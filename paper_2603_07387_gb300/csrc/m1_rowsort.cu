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
constexpr int kRsThreads = 512;  // 16 warps: a strip of 2048 columns
}

// Sorted rows of one (tensor, rep): packed words row << 16 | run end << 15 | negative << 14
// | bin, in the order of the bins (run end: the next row's bin differs, or the last row).
// Counting sort in shared memory (m <= 2^14 counters, n0 <= 2^16 rows).
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
        const uint32_t b = w & mask;
        const int pos = atomicAdd(&cnt[b], 1);
        out[pos] = ((uint32_t)i << 16) | ((w & TNSK_SIGN_BIT) ? (1u << 14) : 0u) | b;
    }
    __syncthreads();
    // run ends: once every row is placed, cnt[b] is the end of bin b's rows, so the row
    // at position k ends its run when k + 1 == cnt[its bin]
    for (int k = threadIdx.x; k < n0; k += blockDim.x) {
        const uint32_t w = out[k];
        if (k + 1 == cnt[w & mask]) out[k] = w | (1u << 15);
    }
}

// One CTA slot: `count` consecutive (strip, sorted row) positions of the concatenation
// over the entries (see M1RowItem). A strip is 2048 columns: each of the 512 lanes owns
// four consecutive columns (one 16-byte load per row; the CTA reads 8 KiB of a row);
// the CTA's warps walk the same rows, whose order words are staged in shared memory
// in chunks of kChunk. A lane's four register sums are added to the shared sketch when
// the row bin changes (the run-end bit of the order word) and at the end of a chunk;
// the shared sketch goes to the entry's global sketch when the walk leaves the entry.
constexpr int kChunk = 512;
constexpr int kCols = 4 * kRsThreads;  // columns of a strip

__global__ void __launch_bounds__(kRsThreads, 2) m1_rowsort_kernel(const M1Tensor* __restrict__ tens,
                                                                   const M1Net* __restrict__ nets,
                                                                   const M1RowSort* __restrict__ rs,
                                                                   const M1RowItem* __restrict__ items,
                                                                   const uint32_t* __restrict__ tabs,
                                                                   const uint32_t* __restrict__ scratch,
                                                                   float* __restrict__ xs) {
    extern __shared__ __align__(16) float x_sh[];  // [max m], then kChunk order words
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
        const int64_t rl = T.numel / n0;  // a multiple of 4 (the planner's condition)
        const float* X = (const float*)T.data;
        const uint32_t* order = scratch + R.order_off;
        uint32_t* s_ord = reinterpret_cast<uint32_t*>(x_sh + ((m + 3) & ~3));
        __syncthreads();  // the previous entry's flush has read x_sh
        for (int b = threadIdx.x; b < m; b += blockDim.x) x_sh[b] = 0.f;
        while (left > 0) {
            // ---- strip `strip`: this lane's four columns, each with its combined word over
            // modes 1 .. order-1 (bins add; the sign bits' sum carries the sign product in bit 24)
            const int64_t c0 = (int64_t)strip * kCols + 4 * threadIdx.x;
            const bool live = c0 < rl;  // all four or none (rl % 4 == 0)
            uint32_t hc[4], cs[4];
            const uint32_t* tab = tabs + N.tab_off + (int64_t)R.rep * N.L;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t wc = 0;
                if (live) {
                    int64_t rem = c0 + j;
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
                hc[j] = wc & mask;
                cs[j] = (wc & TNSK_SIGN_BIT) ? 0x80000000u : 0u;  // the column's sign, as an FP32 sign bit
            }
            const int64_t seg = min(left, n0 - k);  // rows of this strip in the slot
            const float4* Xc = reinterpret_cast<const float4*>(X + c0);
            for (int64_t k1 = k; k1 < k + seg; k1 += kChunk) {
                const int nk = (int)min((int64_t)kChunk, k + seg - k1);
                __syncthreads();  // the previous chunk's words are consumed
                for (int i = threadIdx.x; i < kChunk; i += blockDim.x)
                    s_ord[i] = i < nk ? __ldg(order + k1 + i) : 0u;  // zero words past the end add 0
                __syncthreads();
                float z[4] = {0.f, 0.f, 0.f, 0.f};
                constexpr int kU = 8;  // rows per step: their loads in flight together
                for (int k0 = 0; k0 < nk; k0 += kU) {
                    uint32_t w[kU];
#pragma unroll
                    for (int u = 0; u < kU; u += 4) {
                        const uint4 q = *reinterpret_cast<const uint4*>(s_ord + k0 + u);
                        w[u] = q.x;
                        w[u + 1] = q.y;
                        w[u + 2] = q.z;
                        w[u + 3] = q.w;
                    }
                    float4 v[kU];
#pragma unroll
                    for (int u = 0; u < kU; ++u)
                        v[u] = (live && k0 + u < nk) ? __ldg(Xc + (int64_t)(w[u] >> 16) * (rl >> 2))
                                                     : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const uint32_t rsg = (w[u] << 17) & 0x80000000u;  // the row's sign
                        z[0] += __uint_as_float(__float_as_uint(v[u].x) ^ rsg ^ cs[0]);
                        z[1] += __uint_as_float(__float_as_uint(v[u].y) ^ rsg ^ cs[1]);
                        z[2] += __uint_as_float(__float_as_uint(v[u].z) ^ rsg ^ cs[2]);
                        z[3] += __uint_as_float(__float_as_uint(v[u].w) ^ rsg ^ cs[3]);
                        if (w[u] & (1u << 15)) {  // the bin's run ends here: add the columns' sums
                            if (live) {
                                const uint32_t b = w[u] & mask;
#pragma unroll
                                for (int j = 0; j < 4; ++j) atomicAdd(&x_sh[(b + hc[j]) & mask], z[j]);
                            }
                            z[0] = z[1] = z[2] = z[3] = 0.f;
                        }
                    }
                }
                // a run that continues past the chunk: add its part (the last word read)
                if (live) {
                    const uint32_t b = s_ord[nk - 1] & mask;
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (z[j] != 0.f) atomicAdd(&x_sh[(b + hc[j]) & mask], z[j]);
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
    // the shared sketch (rounded up to 16 bytes), then one chunk of order words
    const size_t smem2 = (size_t)((plan.m1.rs_max_m + 3) & ~3) * 4 + (size_t)kChunk * 4;
    cudaFuncSetAttribute(m1_rowsort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    m1_rowsort_kernel<<<plan.m1.n_rs_items, kRsThreads, smem2, s>>>(tens, nets, rs, items, tabs, scratch, xs);
    return cudaGetLastError();
}

}  // namespace tnsk
