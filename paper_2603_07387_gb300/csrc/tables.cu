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

// (a + b) mod P and (a - b) mod P for a, b < P.
__device__ __forceinline__ uint64_t add61(uint64_t a, uint64_t b) {
    const uint64_t s = a + b;
    return s >= kP61 ? s - kP61 : s;
}
__device__ __forceinline__ uint64_t sub61(uint64_t a, uint64_t b) { return a >= b ? a - b : a + kP61 - b; }

// The sign polynomial c3 x^3 + c2 x^2 + c1 x + c0 mod P at x < 2^32 (Horner).
__device__ __forceinline__ uint64_t sign_poly_u32(const HashCoef& h, uint32_t x) {
    uint64_t g = h.c3;
    g = fold61(mulmod61_u32(g, x) + h.c2);
    g = fold61(mulmod61_u32(g, x) + h.c1);
    return fold61(mulmod61_u32(g, x) + h.c0);
}

// Words of x = x0, x0 + STEP, x0 + 2 STEP, ... (count of them: steps) by forward
// differences, exact in the field mod P: the bin polynomial a1 x + a0 advances by
// STEP a1; the cubic sign polynomial g by its first three differences at x0 (from g at
// x0, x0 + STEP, x0 + 2 STEP) and the constant third difference 6 c3 STEP^3. Four
// modular additions per word instead of four products; the words equal
// hash_packed_u32's. Needs x0 + 2 STEP < 2^32. emit(t, word) stores the word of
// x0 + STEP t.
template <uint32_t STEP = 32, typename Emit>
__device__ __forceinline__ void fd_words(const HashCoef& h, uint32_t x0, int64_t steps, uint32_t mask, Emit emit) {
    uint64_t g = sign_poly_u32(h, x0);
    const uint64_t g1 = sign_poly_u32(h, x0 + STEP), g2 = sign_poly_u32(h, x0 + 2 * STEP);
    uint64_t d1 = sub61(g1, g);
    uint64_t d2 = sub61(add61(g2, g), add61(g1, g1));
    const uint64_t d3 = mulmod61_u32(h.c3, 6u * STEP * STEP * STEP);
    uint64_t b = fold61(mulmod61_u32(h.a1, x0) + h.a0);
    const uint64_t db = mulmod61_u32(h.a1, STEP);
    for (int64_t t = 0; t < steps; ++t) {
        emit(t, (uint32_t)(b & mask) | ((uint32_t)(g & 1) << TNSK_SIGN_SHIFT));
        b = add61(b, db);
        g = add61(g, d1);
        d1 = add61(d1, d2);
        d2 = add61(d2, d3);
    }
}

// Indices [begin, end) of one hash by one warp, lane taking begin + lane + 32 t:
// forward differences where the range is long and below 2^32, else word by word.
template <typename Emit>
__device__ __forceinline__ void warp_words(const HashCoef& h, int64_t begin, int64_t end, uint32_t mask, int lane,
                                           Emit emit) {
    const int64_t x0 = begin + lane;
    if (end - begin >= 256 && x0 + 64 < (1ll << 32)) {
        const int64_t steps = x0 < end ? (end - x0 + 31) / 32 : 0;
        const int64_t lim = ((1ll << 32) - x0 + 31) / 32;  // words below 2^32: the 32-bit form
        fd_words(h, (uint32_t)x0, steps < lim ? steps : lim, mask,
                 [&](int64_t t, uint32_t w) { emit(x0 + 32 * t, w); });
        for (int64_t i = x0 + 32 * lim; i < end; i += 32) emit(i, hash_packed(h, (uint64_t)i, mask));
        return;
    }
    for (int64_t i = x0; i < end; i += 32)
        emit(i, i < (1ll << 32) ? hash_packed_u32(h, (uint32_t)i, mask) : hash_packed(h, (uint64_t)i, mask));
}

// Table rows (request, rep) in contiguous ranges per warp, 32 rows at a time: lane j
// finds row j's request (advancing from the previous row's) and derives its SplitMix64
// key chain and six polynomial coefficients, so each lane pays for one row's setup;
// then the warp writes the rows one after another, the row's coefficients broadcast
// from its lane, lanes over the row's indices (coalesced stores).
__global__ void __launch_bounds__(256) draw_tables_kernel(const TabReq* __restrict__ reqs, int nreq, int64_t rows,
                                                          uint32_t* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t per = (rows + nwarps - 1) / nwarps;
    const int64_t r0 = warp * per, r1 = r0 + per < rows ? r0 + per : rows;
    if (r0 >= r1) return;
    int k = find_req(reqs, nreq, r0, [](const TabReq& r) { return r.crow; });
    for (int64_t g0 = r0; g0 < r1; g0 += 32) {
        const int64_t row = g0 + lane;
        int kk = k;
        while (kk + 1 < nreq && reqs[kk + 1].crow <= row) ++kk;
        k = __shfl_sync(0xffffffffu, kk, 31);
        HashCoef hc{0, 0, 0, 0, 0, 0};
        unsigned long long dst_l = 0;
        long long n_l = 0;
        uint32_t mask_l = 0;
        if (row < r1) {
            const TabReq& q = reqs[kk];
            const uint64_t rep = (uint64_t)(row - q.crow);
            hc = hash_coef(q.seed, (uint64_t)q.rep_base + rep, q.tid);
            dst_l = (unsigned long long)(uintptr_t)(out + q.out_off + (int64_t)rep * q.rep_stride);
            n_l = q.n;
            mask_l = q.mask;
        }
        const int cnt = r1 - g0 < 32 ? (int)(r1 - g0) : 32;
        // short rows (at most 32 indices, e.g. the bonds and legs of small networks): each
        // lane writes its own row by forward differences of step 1, instead of the warp
        // taking the rows one after another with most lanes idle
        if (__all_sync(0xffffffffu, row >= r1 || n_l <= 32)) {
            if (row < r1 && n_l > 0) {
                uint32_t* dst = (uint32_t*)(uintptr_t)dst_l;
                if (n_l >= 4)
                    fd_words<1>(hc, 0u, n_l, mask_l, [&](int64_t t, uint32_t w) { dst[t] = w; });
                else
                    for (int x = 0; x < (int)n_l; ++x) dst[x] = hash_packed_u32(hc, (uint32_t)x, mask_l);
            }
            continue;
        }
        for (int i = 0; i < cnt; ++i) {
            HashCoef h;
            h.a0 = __shfl_sync(0xffffffffu, (unsigned long long)hc.a0, i);
            h.a1 = __shfl_sync(0xffffffffu, (unsigned long long)hc.a1, i);
            h.c0 = __shfl_sync(0xffffffffu, (unsigned long long)hc.c0, i);
            h.c1 = __shfl_sync(0xffffffffu, (unsigned long long)hc.c1, i);
            h.c2 = __shfl_sync(0xffffffffu, (unsigned long long)hc.c2, i);
            h.c3 = __shfl_sync(0xffffffffu, (unsigned long long)hc.c3, i);
            uint32_t* dst = (uint32_t*)(uintptr_t)__shfl_sync(0xffffffffu, dst_l, i);
            const int64_t n = __shfl_sync(0xffffffffu, n_l, i);
            const uint32_t mask = __shfl_sync(0xffffffffu, mask_l, i);
            warp_words(h, 0, n, mask, lane, [&](int64_t x, uint32_t w) { dst[x] = w; });
        }
    }
}

// One hash over [0, n): each warp a contiguous range of indices (a multiple of 32).
__global__ void __launch_bounds__(256) count_sketch_kernel(uint64_t seed, uint64_t rep, uint64_t tid, int64_t n,
                                                           uint32_t mask, int32_t* __restrict__ bins,
                                                           int8_t* __restrict__ signs) {
    const HashCoef h = hash_coef(seed, rep, tid);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t per = ((n + nwarps - 1) / nwarps + 31) & ~(int64_t)31;
    const int64_t begin = warp * per;
    if (begin >= n) return;
    const int64_t end = begin + per < n ? begin + per : n;
    warp_words(h, begin, end, mask, threadIdx.x & 31, [&](int64_t i, uint32_t w) {
        bins[i] = (int32_t)(w & mask);
        signs[i] = (w & TNSK_SIGN_BIT) ? (int8_t)-1 : (int8_t)1;
    });
}

cudaError_t launch_draw_tables(const TabReq* d_reqs, int nreq, int64_t rows, uint32_t* d_out, cudaStream_t s) {
    if (rows <= 0 || nreq <= 0) return cudaSuccess;
    // 8 warps per block, a few rows per warp: enough warps to hide the latency of the
    // word recurrences
    int64_t blocks = (rows + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    draw_tables_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_reqs, nreq, rows, d_out);
    return cudaGetLastError();
}

cudaError_t launch_count_sketch(uint64_t seed, uint64_t rep, uint64_t tid, int64_t n, int64_t m, int32_t* bins,
                                int8_t* signs, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 2047) / 2048;  // 8 warps of at least 256 indices
    if (blocks > 152 * 8) blocks = 152 * 8;
    count_sketch_kernel<<<(unsigned)blocks, 256, 0, s>>>(seed, rep, tid, n, (uint32_t)(m - 1), bins, signs);
    return cudaGetLastError();
}

}  // namespace tnsk
