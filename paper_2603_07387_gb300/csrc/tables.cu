// tables.cu -- row a1 of the hot path: draw the count sketches of every
// repetition (Sec. 2.1 Def. "Count sketch"; Alg. 1 "C_u independent count
// sketch"; Alg. 2 "independent recursive sketch" R_k) as packed table words.
#include "kernels.cuh"

namespace tnsk {

// Finds the request holding flat position g of a prefix array (binary search).
template <typename F>
__device__ __forceinline__ int find_req(const TabReq* __restrict__ reqs, int nreq, int64_t g, F key) {
    int lo = 0, hi = nreq - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (key(reqs[mid]) <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// One warp per table row (request, rep): the SplitMix64 key chain and the six
// polynomial coefficients once per row, then the lanes over the row's indices
// (coalesced stores). Warps stride over the rows of all requests.
__global__ void __launch_bounds__(256) draw_tables_kernel(const TabReq* __restrict__ reqs, int nreq, int64_t rows,
                                                          uint32_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += nwarps) {
        const TabReq& q = reqs[find_req(reqs, nreq, row, [](const TabReq& r) { return r.crow; })];
        const uint64_t rep = (uint64_t)(row - q.crow);
        const HashCoef h = hash_coef(q.seed, (uint64_t)q.rep_base + rep, q.tid);
        uint32_t* dst = out + q.out_off + (int64_t)rep * q.rep_stride;
        const int64_t n32 = q.n < (1ll << 32) ? q.n : (1ll << 32);
        for (int64_t i = lane; i < n32; i += 32) dst[i] = hash_packed_u32(h, (uint32_t)i, q.mask);
        for (int64_t i = n32 + lane; i < q.n; i += 32) dst[i] = hash_packed(h, (uint64_t)i, q.mask);
    }
}

__global__ void count_sketch_kernel(uint64_t seed, uint64_t rep, uint64_t tid, int64_t n, uint32_t mask,
                                    int32_t* __restrict__ bins, int8_t* __restrict__ signs) {
    HashCoef h = hash_coef(seed, rep, tid);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t w = hash_packed(h, (uint64_t)i, mask);
        bins[i] = (int32_t)(w & mask);
        signs[i] = (w & TNSK_SIGN_BIT) ? (int8_t)-1 : (int8_t)1;
    }
}

cudaError_t launch_draw_tables(const TabReq* d_reqs, int nreq, int64_t rows, uint32_t* d_out, cudaStream_t s) {
    if (rows <= 0 || nreq <= 0) return cudaSuccess;
    int64_t blocks = (rows + 7) / 8;  // 8 warps per block, one row each per pass
    if (blocks > 152 * 16) blocks = 152 * 16;
    draw_tables_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_reqs, nreq, rows, d_out);
    return cudaGetLastError();
}

cudaError_t launch_count_sketch(uint64_t seed, uint64_t rep, uint64_t tid, int64_t n, int64_t m, int32_t* bins,
                                int8_t* signs, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    count_sketch_kernel<<<(unsigned)blocks, 256, 0, s>>>(seed, rep, tid, n, (uint32_t)(m - 1), bins, signs);
    return cudaGetLastError();
}

}  // namespace tnsk
