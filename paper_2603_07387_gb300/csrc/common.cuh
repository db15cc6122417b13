// common.cuh -- shared device helpers and launch descriptors of libtnsk.
//
// Everything here is GPU-path code; the CPU oracle implements the same hash
// contract independently and shares nothing with this file.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tnsk.h"

#define TNSK_MAX_ORDER 12
#define TNSK_MAX_M (1 << 16)
#define TNSK_SIGN_SHIFT 24  // packed table word: bin in bits [0,24), sign in bit 24
#define TNSK_SIGN_BIT (1u << TNSK_SIGN_SHIFT)

namespace tnsk {

// ---------------------------------------------------------------------------
// Hash contract (Sec. 2.1 Def. "Count sketch"; construction fixed by tnsk.h)
// ---------------------------------------------------------------------------
constexpr uint64_t kP61 = 0x1FFFFFFFFFFFFFFFull;

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t state) {
    uint64_t z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// x mod P for any 64-bit x (2^61 = 1 mod P).
__device__ __forceinline__ uint64_t fold61(uint64_t x) {
    uint64_t r = (x & kP61) + (x >> 61);
    return r >= kP61 ? r - kP61 : r;
}

// (a * b) mod P for a, b < P: 2^64 = 8 (mod P), so hi*2^64 + lo = 8 hi + lo.
__device__ __forceinline__ uint64_t mulmod61(uint64_t a, uint64_t b) {
    uint64_t lo = a * b;
    uint64_t hi = __umul64hi(a, b);
    return fold61((lo & kP61) + (lo >> 61) + (hi << 3));
}

struct HashCoef {
    uint64_t a0, a1, c0, c1, c2, c3;
};

__device__ __forceinline__ HashCoef hash_coef(uint64_t seed, uint64_t rep, uint64_t tid) {
    uint64_t key = splitmix64(splitmix64(splitmix64(seed) ^ rep) ^ tid);
    HashCoef h;
    h.a0 = fold61(splitmix64(key ^ 0));
    h.a1 = fold61(splitmix64(key ^ 1));
    h.c0 = fold61(splitmix64(key ^ 8));
    h.c1 = fold61(splitmix64(key ^ 9));
    h.c2 = fold61(splitmix64(key ^ 10));
    h.c3 = fold61(splitmix64(key ^ 11));
    return h;
}

// (a * x) mod P for a < P and x < 2^32: with a = ah 2^32 + al,
// a x = ah x 2^32 + al x, and ah x 2^32 = (ah x mod 2^29) 2^32 + (ah x >> 29) 2^61
// with 2^61 = 1 (mod P); two 32 x 32 -> 64-bit products instead of a 64 x 64 one.
__device__ __forceinline__ uint64_t mulmod61_u32(uint64_t a, uint32_t x) {
    const uint64_t p1 = (uint64_t)(uint32_t)(a >> 32) * x;  // < 2^61
    const uint64_t p0 = (uint64_t)(uint32_t)a * x;          // < 2^64
    return fold61((p0 & kP61) + (p0 >> 61) + ((p1 & 0x1FFFFFFFull) << 32) + (p1 >> 29));
}

// hash_packed for an index below 2^32 (x = i < P needs no reduction).
__device__ __forceinline__ uint32_t hash_packed_u32(const HashCoef& h, uint32_t x, uint32_t mask) {
    const uint64_t b = fold61(mulmod61_u32(h.a1, x) + h.a0);
    uint64_t g = h.c3;
    g = fold61(mulmod61_u32(g, x) + h.c2);
    g = fold61(mulmod61_u32(g, x) + h.c1);
    g = fold61(mulmod61_u32(g, x) + h.c0);
    return (uint32_t)(b & mask) | ((uint32_t)(g & 1) << TNSK_SIGN_SHIFT);
}

// Packed table word for index i: bin | (negative sign) << 24. m is a power of two.
__device__ __forceinline__ uint32_t hash_packed(const HashCoef& h, uint64_t i, uint32_t mask) {
    uint64_t x = fold61(i);
    uint64_t b = fold61(mulmod61(h.a1, x) + h.a0);
    uint64_t g = h.c3;
    g = fold61(mulmod61(g, x) + h.c2);
    g = fold61(mulmod61(g, x) + h.c1);
    g = fold61(mulmod61(g, x) + h.c0);
    return (uint32_t)(b & mask) | ((uint32_t)(g & 1) << TNSK_SIGN_SHIFT);
}

__host__ __device__ __forceinline__ uint64_t tid_m1_edge(int e) { return (1ull << 56) | (uint64_t)e; }
__host__ __device__ __forceinline__ uint64_t tid_m2_edge(int e) { return (2ull << 56) | (uint64_t)e; }
__host__ __device__ __forceinline__ uint64_t tid_m2_pad(int k, int j) {
    return (3ull << 56) | ((uint64_t)k << 24) | (uint64_t)j;
}
__host__ __device__ __forceinline__ uint64_t tid_m2_ts(int k, int lam, int j, int s) {
    return (4ull << 56) | ((uint64_t)k << 24) | ((uint64_t)lam << 16) | ((uint64_t)j << 1) | (uint64_t)s;
}

// ---------------------------------------------------------------------------
// Table draw requests (row a1 of the hot path)
// ---------------------------------------------------------------------------
struct TabReq {
    uint64_t seed;
    uint64_t tid;
    int64_t n;          // domain size
    int64_t out_off;    // packed-table offset of rep 0
    int64_t rep_stride; // distance between consecutive reps
    int64_t crow;       // first table row of this request (prefix over R)
    int64_t rep_base;   // repetition index of the request's first row (tnsk_params.rep0)
    int32_t R;
    uint32_t mask;      // m - 1
};

// ---------------------------------------------------------------------------
// Input loads
// ---------------------------------------------------------------------------
template <typename AccT>
__device__ __forceinline__ AccT load_as(const void* p, int dtype, int64_t i) {
    if (dtype == TNSK_F32) return (AccT)__ldg((const float*)p + i);
    if (dtype == TNSK_F64) return (AccT)__ldg((const double*)p + i);
    return (AccT)__bfloat162float(((const __nv_bfloat16*)p)[i]);
}

// ---------------------------------------------------------------------------
// Method 1 descriptors
// ---------------------------------------------------------------------------
struct M1Tensor {
    const void* data;
    int64_t numel;
    int64_t O;                           // product of the tensor's open dims
    int64_t xoff;                        // offset of its [O][m] block in one rep's sketches
    int64_t soff;                        // open spectra block in one rep's spectra (-1: folded into P)
    int64_t eoff;                        // exponents of those spectra in one rep's exponent block
    int64_t ostride[TNSK_MAX_ORDER];     // open-index stride of each mode (0 if contracted)
    int32_t dims[TNSK_MAX_ORDER];
    int32_t tab[TNSK_MAX_ORDER];         // offset of the mode's table in the rep block, -1 if open
    int32_t comp[TNSK_MAX_ORDER];        // 1: second mode of its edge (complement)
    int32_t dtype;
    int32_t order;
    int32_t net;
    int32_t n_ctr;                       // contracted modes
};

#define TNSK_MAX_OPEN_TENSORS 4

// A diagonal copy tensor delta(i, ..., i) of WLOG 1 (Sec. 4.1), never stored: its n
// nonzeros are sketched directly (every mode contracted, all at index i).
struct M1Diag {
    int32_t tensor;  // index into the method-1 tensor descriptors
    int32_t net;     // index into the method-1 network descriptors
    int64_t n;
};

// Row-sorted sketch of one (tensor, rep) (m1_rowsort.cu): the tensor's rows in the order
// of their leading-mode bins, packed row << 15 | negative << 14 | bin, at order_off
// (words) in the plan's scratch.
struct M1RowSort {
    int32_t tensor;  // index into the method-1 tensor descriptors
    int32_t net;     // index into the method-1 network descriptors
    int32_t rep;     // repetition within the call
    int32_t strips;  // column strips of 2048
    int64_t order_off;
};

// One CTA of the row-sorted sketch: `count` consecutive (strip, sorted row) positions of
// the concatenation over all M1RowSort entries (strips in order, sorted rows within a
// strip), starting at row k of strip `strip` of entry rs. The planner splits the whole
// concatenation into one equal part per CTA slot.
struct M1RowItem {
    int32_t rs, strip, k;
    int32_t pad_;
    int64_t count;
};

struct M1Net {
    int64_t m;
    int64_t L;        // table words per rep
    int64_t tab_off;  // packed tables of rep 0
    int64_t X;        // sketch entries per rep
    int64_t x_off;    // sketch buffer offset of rep 0
    int64_t O;        // output entries
    int64_t y_off;    // per-rep estimate buffer offset [R][O]
    int64_t spec_off; // open-tensor spectra of rep 0 (complex entries)
    int64_t spec_per_rep;
    int64_t exp_off;  // their exponents (ints) of rep 0
    int64_t exp_per_rep;
    int64_t lspec_off;  // spectra of rep 0: [R][p][m/2] (large m, pass-1 output) or [R][p][m/2 + 1] (mid m), complex
    int64_t yabs_off;   // per-rep magnitude sums (1/m) sum_j (|Re| + |Im|)(prod_k F x_k(j)) [R] (networks without
                        // open legs), in the per-rep estimate buffer after all estimates
    int32_t log2m;
    int32_t R;
    int32_t t0;       // first tensor
    int32_t p;
    int32_t open0;    // first entry in the open-mode list
    int32_t n_open;
    int32_t groups;
    int32_t n_ot;     // tensors with O > 1 ("open tensors")
    int32_t ot[TNSK_MAX_OPEN_TENSORS];
    double* out;      // combined estimate [O]
    double* per_rep;  // optional user copy [R][O]
};

struct OpenMode {      // output mode j of a network
    int64_t ostride;   // stride in the output index (row-major over the open list)
    int64_t tstride;   // stride in its tensor's open index
    int32_t dim;
    int32_t slot;      // open-tensor slot of the owning tensor
};

struct M1Work {
    int64_t begin, end;  // entry range of the tensor
    int32_t tensor;
    int32_t rep0;
    int32_t nrep;
    int32_t priv;        // 0: global atomics; 1: shared-memory bins flushed by atomics;
                         // 2: shared-memory bins of a whole tensor, flushed by stores
    int32_t gtab;        // 1: hash-table words read from global memory (large tables),
                         // 0: staged in shared memory
    int32_t ltab;        // staged tables hold only the index range of each mode that
                         // [begin, end) touches (large tensors sketched in chunks)
};

template <typename T>
struct alignas(2 * sizeof(T)) Cplx {
    T x, y;
};

// ---------------------------------------------------------------------------
// Error word written by kernels (bounds / waits); read back by tnsk_sync.
// ---------------------------------------------------------------------------
enum : int { DEVERR_NONE = 0, DEVERR_BOUNDS = 1, DEVERR_TIMEOUT = 2 };

}  // namespace tnsk
