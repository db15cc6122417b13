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

// The polynomial coefficients of every (request, rep): the SplitMix64 key chain
// runs once per table instead of once per word.
__global__ void table_coef_kernel(const TabReq* __restrict__ reqs, int nreq, int64_t rows, HashCoef* __restrict__ coef) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < rows; g += (int64_t)gridDim.x * blockDim.x) {
        const int q = find_req(reqs, nreq, g, [](const TabReq& r) { return r.crow; });
        const TabReq& t = reqs[q];
        coef[g] = hash_coef(t.seed, (uint64_t)(g - t.crow), t.tid);
    }
}

// One thread per table word.
__global__ void draw_tables_kernel(const TabReq* __restrict__ reqs, int nreq, int64_t total,
                                   const HashCoef* __restrict__ coef, uint32_t* __restrict__ out) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int qi = find_req(reqs, nreq, g, [](const TabReq& r) { return r.first; });
        const TabReq& q = reqs[qi];
        const uint64_t local = (uint64_t)(g - q.first);
        uint64_t rep, i;
        if (local < (1ull << 32) && q.n < (1ll << 32)) {
            const uint32_t r32 = (uint32_t)local / (uint32_t)q.n;
            rep = r32;
            i = (uint32_t)local - r32 * (uint32_t)q.n;
        } else {
            rep = local / (uint64_t)q.n;
            i = local - rep * (uint64_t)q.n;
        }
        const HashCoef h = coef[q.crow + rep];
        out[q.out_off + rep * q.rep_stride + i] = hash_packed(h, (uint64_t)i, q.mask);
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

cudaError_t launch_draw_tables(const TabReq* d_reqs, int nreq, int64_t total, int64_t rows, HashCoef* d_coef,
                               uint32_t* d_out, cudaStream_t s) {
    if (total <= 0 || nreq <= 0) return cudaSuccess;
    int64_t cblocks = (rows + 127) / 128;
    if (cblocks > 152 * 16) cblocks = 152 * 16;
    table_coef_kernel<<<(unsigned)cblocks, 128, 0, s>>>(d_reqs, nreq, rows, d_coef);
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    draw_tables_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_reqs, nreq, total, d_coef, d_out);
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
