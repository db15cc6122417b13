// method2.cuh -- descriptors of method 2 (Sec. 4.4, Eq. 2, Alg. 2, 4, 5).
//
// The rooted tree is evaluated by height (leaves first). Per repetition r every
// non-root tensor k produces x_k = C_{par,k} mat(X_k) R_k^T r_k (an m-vector;
// Alg. 5), every tensor with children produces r_k = Q_k((x) x_l) (Alg. 2
// NeighborsSketch), and the root gives y_r = x_o^T r_o = sum_i X_o(i) sigma(i)
// r_o[b(i)] with (sigma, b) of R_o from Alg. 4.
//
// GPU layout (per batch, in the scratch arena):
//   tables   per network and rep: [edge tables C_{k,l} (sum n_e words)]
//            [padding-slot words (sum_k qt_k)] [T_{l,j} tables (2(qt_k-1) m words per k)]
//   x        per non-root node: [R][m] accumulators (zeroed per call)
//   r        per node with >= 2 children: [R][(qt-1) m] level outputs; the last
//            m-vector of each rep is r_k
//   V        per node with children: [R][cols]: V(col, r) = sigma_r(col) r_k[r][b_r(col)],
//            so that x_k = scatter_C( mat(X_k) V ) is a matrix product batched over reps
//   W^T      FP32 tensor-core path: [R][npar] the product before the scatter (zeroed)
//   y        per root: [R] FP64 accumulators
#pragma once

#include <string>
#include <vector>

#include "common.cuh"

namespace tnsk {

// Splits an FP32 value into two TF32 values with x = hi + lo up to the rounding
// of lo: each part rounded to nearest, ties away from zero, by adding half a
// TF32 unit in the last place to the bit pattern and clearing the 13 low bits
// (a carry into the exponent is the correct rounding up). Integer operations
// only, so the split of a streamed operand does not queue on the conversion
// unit. x - hi is exact in FP32 (hi is within a factor of two of x).
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
    hi = (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
    lo = (__float_as_uint(x - __uint_as_float(hi)) + 0x1000u) & 0xFFFFE000u;
}

#define TNSK_MAX_SLOTS 16  // slots of a recursive sketch: children padded to a power of two

struct M2Node {
    const void* data;
    int64_t numel;
    int64_t A;        // X viewed as [A][npar][Bc]: modes before / the parent mode / after
    int64_t npar;     // parent-mode dim (1 for the root)
    int64_t Bc;
    int64_t cols;     // A * Bc: product of the child-mode dims
    int64_t ptab;     // parent edge table offset in a rep's table block (-1: root)
    int64_t ctab[TNSK_MAX_ORDER];  // child slot j: its edge table offset
    int64_t pad_tab;  // offset of this node's padding words (slot j at pad_tab + j)
    int64_t t_tab;    // offset of this node's T tables
    int64_t x_off;    // [R][m] sketch accumulators of this (non-root) node, -1 for the root
    int64_t r_off;    // [R][(qt-1) m] composition outputs (qt >= 2), else -1
    int64_t src_off;  // r_k used by V: r_off + (qt-2) m for qt >= 2, the child's x_off for qt = 1
    int64_t src_stride;  // distance between reps in the r_k source
    int64_t v_off;    // [R][cols] V matrix (nodes with children); FP32 non-root nodes hold the
                      // TF32 hi part there and the lo part in the next [R][cols]
    int64_t w_off;    // tensor-core path: [R][npar] product W^T = (mat(X_k) V)^T, -1 otherwise
    int64_t child_x[TNSK_MAX_SLOTS];  // slot j < c: the child's x_off
    int32_t dims[TNSK_MAX_ORDER];
    int32_t cmode[TNSK_MAX_ORDER];    // slot j < c: this node's mode toward child j
    int32_t dtype;
    int32_t order;
    int32_t pmode;    // parent mode (-1 root)
    int32_t c;        // children
    int32_t qt;       // slots (0 for a leaf)
    int32_t net;      // method-2 network index
    int32_t is_root;
    int32_t tm_x;     // streaming tensor-core path: tensor-map index of X and of V^T
    int32_t tm_v;
    int32_t r_fact;   // grouped tensor in factored form: 1 SIMT (M2_GEMM_RUNGF), 2 tensor
                      // cores (M2_GEMM_RUNGT, factors prepared at rc_off)
    int32_t vbf16;    // BF16 product (M2_GEMM_BF16): V^T stored as three BF16 parts
                      // [3][R][cols] at byte offset 4 v_off, X maps tm_x, parts tm_v .. + 2
    // grouped (rung) tensor, M2_GEMM_RUNG: X(row, col) = sum_s A[i1 ai + j1 aj + s as]
    // B[i2 bi + j2 bj + s bs] with row = i1 rn_i2 + i2, col = j1 rn_j2 + j2
    const float* rA;
    const float* rB;
    int32_t rn_i1, rn_i2, rn_j1, rn_j2, rs;
    int32_t r_ai, r_aj, r_as, r_bi, r_bj, r_bs;
    int32_t r_astage;  // 1: the tile's A rows are staged in shared memory after B
    int64_t rc_off;    // M2_GEMM_RUNGT: TF32 hi / lo parts of B and A, [Bh | Bl | Ah | Al] of
                       // rs 1024 floats each (m2_rung_prep_kernel), -1 otherwise
};

struct M2Net {
    int64_t m;
    int64_t Lrep;     // table words per rep
    int64_t tab_off;  // table block of rep 0
    int64_t y_off;    // per-rep estimates [R] (FP64), inside the shared [R][O] buffer
    int32_t log2m;
    int32_t R;
};

// Work items (node index into the batch's node array + a chunk of its work).
struct M2Item {
    int32_t node;
    int32_t a;        // first rep (compose) or row tile (gemm) or chunk index
    int32_t b;        // rep tile (gemm)
    int32_t pad_;     // tensor-core gemm: index of this item's K split
    int64_t begin, end;  // element range (leaf / vbuild / root chunks); tensor-core gemm:
                         // begin = number of K splits
};

// M2_GEMM_STREAM: tensor-core tiles of row-major FP32 tensors with contiguous
// rows (parent mode first, 4 | cols, 16-byte aligned): streaming kernel.
// M2_WSCATTER: x_k[r][h(i)] += s(i) W^T[r][i] for the tensor-core tiles.
enum M2Kind {
    M2_LEAF = 0,
    M2_COMPOSE = 1,
    M2_VBUILD = 2,
    M2_GEMM = 3,
    M2_GEMM_STREAM = 4,
    M2_GEMM_RUNG = 5,
    M2_GEMM_RUNGF = 6,  // grouped tensor in factored form (dims <= 32): it.a first rep, it.b reps
    M2_GEMM_BF16 = 7,   // TNSK_PREC_BF16: BF16 tensors on the kind::f16 tensor-core kernel
    M2_GEMM_RUNGT = 8,  // grouped tensor in factored form on the tensor cores (factor dims 32,
                        // s <= 8): it.a first rep, it.b reps (<= 4); one persistent launch
    M2_WSCATTER = 9,
    M2_ROOT = 10,
    M2_RUNG_PREP = 11,  // the prepared factors of every M2_GEMM_RUNGT node (height 0)
    M2_NKINDS = 12
};

struct M2Plan {
    int n_nets = 0;
    size_t nodes_off = 0, nets_off = 0, items_off = 0;
    size_t ws_off = 0;  // x / r / V / y workspace base (all offsets above are relative to it)
    int max_height = -1;
    bool idx32 = true;  // every node has fewer than 2^32 columns
    int max_qt = 0;     // largest slot count
    int max_order = 0;  // largest tensor order
    size_t tmaps_off = 0;  // tensor maps (128 B each) in the descriptor block
    size_t scatter_smem = 0;  // shared-memory bins of the largest row-scatter item
    size_t vbuild_smem = 0;   // staged T tables + child sketches of the largest staged V-build item
    size_t rung_smem = 0;     // dynamic shared memory of the grouped-tensor GEMM (V ring + B)
    size_t rungf_smem = 0;    // dynamic shared memory of the factored grouped-tensor product
    // tensor maps to encode once the device addresses are fixed: node, 0 = X / 1 = V^T hi / 2 = lo
    std::vector<std::pair<int, int>> tmap_jobs;
    int max_log2m = 0;
    // per height, per kind: [first, count) into the item array
    std::vector<int> first, count;  // size (max_height+1) * M2_NKINDS
};

struct BatchPlan;
struct Profiler;
// inject (tests only, tnsk_debug_inject): the tensor-core products' TMA producers issue
// no loads, so their consumers' bounded waits run out and report DEVERR_TIMEOUT
tnsk_status run_method2(const BatchPlan& plan, unsigned char* base, bool fp64, const void* const* d_tws,
                        cudaStream_t s, Profiler& prof, int* d_err, std::string& err, int inject = 0);
cudaError_t launch_m2_gemm_tc(int n, const M2Node* nodes, const M2Net* nets, const M2Item* items,
                              const uint32_t* tabs, float* ws, const unsigned char* tmaps, int* err, bool stream,
                              int inject, cudaStream_t s);
// BF16 tiles (M2_GEMM_BF16): X and the three BF16 parts of V^T by TMA, kind::f16.
cudaError_t launch_m2_gemm_bf16(int n, const M2Node* nodes, const M2Net* nets, const M2Item* items, float* ws,
                                const unsigned char* tmaps, int* err, int inject, cudaStream_t s);
// Grouped-tensor tiles (M2_GEMM_RUNG); smem from m2_gemm_rung_smem(bytes of the staged B).
size_t m2_gemm_rung_smem(size_t b_bytes);
cudaError_t launch_m2_gemm_tc_rung(int n, const M2Node* nodes, const M2Net* nets, const M2Item* items, float* ws,
                                   const unsigned char* tmaps, int* err, size_t smem, cudaStream_t s);
// Grouped tensors with every factor dim <= 32 (M2_GEMM_RUNGF): the product in factored
// form, SIMT FP32; smem from m2_rung_fact_smem(s).
size_t m2_rung_fact_smem(int s);
cudaError_t launch_m2_rung_fact(int n, const M2Node* nodes, const M2Net* nets, const M2Item* items, float* ws,
                                size_t smem, cudaStream_t s);
// Grouped tensors with all four factor dims 32 and s <= 8 (M2_GEMM_RUNGT): the factored
// product on the tensor cores, one persistent CTA per SM over the n blocks; the factors'
// TF32 parts first by launch_m2_rung_prep (one block per item of M2_RUNG_PREP).
cudaError_t launch_m2_rung_prep(int n, const M2Node* nodes, const M2Item* items, float* ws, cudaStream_t s);
cudaError_t launch_m2_rung_tc(int n, const M2Node* nodes, const M2Item* items, float* ws, const unsigned char* tmaps,
                              int* err, int inject, cudaStream_t s);

}  // namespace tnsk
