// m2_rung_fact.cu -- method 2's sketched product (row a7, Alg. 5) for a grouped
// tensor in factored form, so its entries are never formed.
//
// A grouped (rung) tensor is X((i1,i2),(j1,j2)) = sum_s A(i1,s,j1) B(i2,s,j2) (the
// exact grouping of Sec. 4.1, indices named by the node's row / column split). The
// product W^T[r][(i1,i2)] = sum_{j1,j2} X((i1,i2),(j1,j2)) V[r][(j1,j2)] is taken as
//   U_s[i2][j1] = sum_{j2} B(i2,s,j2) V_r[j1][j2]         (one 32x32x32 product per s)
//   W_r[i1][i2] = sum_s sum_{j1} A(i1,s,j1) U_s[i2][j1]   (one 32x32x32 product per s)
// which costs 2 s n^3 multiply-adds per rep for n = 32 instead of the n^4 of the
// dense product, and reads A and B (s n^2 values each) instead of X (n^4).
//
// One CTA (8 warps) per (node, block of reps): A and B are staged in shared memory
// once by asynchronous copies, as [s][32][32] tiles (zero outside the node's dims, so any dims up to 32
// work); per rep V_r = hi + lo of the V build's TF32 split is staged as [j1][j2]
// (double-buffered: the next rep's V is loaded into registers during this rep);
// warp w takes s = w, w + 8, ...: U_s into its own tile, then its partial W from it,
// both by the same register-blocked SIMT product (lane: 4 rows x 8 columns, K in
// float4 steps; tiles XOR-swizzled by 16-byte chunks so the float4 loads of 8
// consecutive rows fall in different banks). The 8 partial W tiles are summed and
// stored as the rep's W^T row (plain stores: the whole row is written), FP32.
#include <algorithm>

#include "method2.cuh"

namespace tnsk {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kTile = 32 * 32;

// Offset of (row, col) in a 32 x 32 FP32 tile whose 16-byte chunks are swizzled by row.
__device__ __forceinline__ int swz(int row, int col) { return row * 32 + ((((col >> 2) ^ (row & 7)) << 2) | (col & 3)); }

// c[i][j] += sum_k P[ab + 8 i][k] Q[bb + 4 j][k], k < 32, on swizzled tiles (plain
// fmaf: measured faster here than packed pairs).
__device__ __forceinline__ void tile_nt(const float* __restrict__ P, const float* __restrict__ Q, int ab, int bb,
                                        float (&c)[4][8]) {
#pragma unroll 1
    for (int k4 = 0; k4 < 8; ++k4) {
        float4 p[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)  // rows ab + 8 i share row & 7 = ab
            p[i] = *reinterpret_cast<const float4*>(P + (ab + 8 * i) * 32 + ((k4 ^ ab) << 2));
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int row = bb + 4 * j;
            const float4 q = *reinterpret_cast<const float4*>(Q + row * 32 + ((k4 ^ (row & 7)) << 2));
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float t = c[i][j];
                t = fmaf(p[i].x, q.x, t);
                t = fmaf(p[i].y, q.y, t);
                t = fmaf(p[i].z, q.z, t);
                t = fmaf(p[i].w, q.w, t);
                c[i][j] = t;
            }
        }
    }
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 2) m2_rung_fact_kernel(const M2Node* __restrict__ nodes,
                                                                  const M2Net* __restrict__ nets,
                                                                  const M2Item* __restrict__ items,
                                                                  float* __restrict__ ws) {
    extern __shared__ __align__(16) float sm[];
    const M2Item it = items[blockIdx.x];
    const M2Node& nd = nodes[it.node];
    const M2Net& N = nets[nd.net];
    const int S = nd.rs;
    const int n_i1 = nd.rn_i1, n_i2 = nd.rn_i2, n_j1 = nd.rn_j1, n_j2 = nd.rn_j2;
    float* sA = sm;                       // [S][32 x 32]: A(i1, s, j1) at [s][i1][j1]
    float* sB = sA + (size_t)S * kTile;   // [S][32 x 32]: B(i2, s, j2) at [s][i2][j2]
    float* sV = sB + (size_t)S * kTile;   // [2][32 x 32]: V_r at [j1][j2], double-buffered
    float* sU = sV + 2 * kTile;           // [8][32 x 32]: per warp U_s, then its partial W
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ab = lane >> 2, bb = lane & 3;
    {
        // A and B into shared memory by asynchronous 4-byte copies (all in flight at
        // once; entries outside the dims are zero-filled: source size 0)
        const float* __restrict__ gA = nd.rA;
        const float* __restrict__ gB = nd.rB;
        const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm);
        for (int e = tid; e < S * kTile; e += kThreads) {
            const int s = e >> 10, row = (e >> 5) & 31, col = e & 31;
            const bool ia = row < n_i1 && col < n_j1, ib = row < n_i2 && col < n_j2;
            const float* pa = ia ? gA + (int64_t)row * nd.r_ai + (int64_t)col * nd.r_aj + (int64_t)s * nd.r_as : gA;
            const float* pb = ib ? gB + (int64_t)row * nd.r_bi + (int64_t)col * nd.r_bj + (int64_t)s * nd.r_bs : gB;
            const uint32_t da = sbase + (uint32_t)(s * kTile + swz(row, col)) * 4u;
            const uint32_t db = da + (uint32_t)(S * kTile) * 4u;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(da), "l"(pa), "r"(ia ? 4 : 0)
                         : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(db), "l"(pb), "r"(ib ? 4 : 0)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    const int64_t R = N.R, npar = nd.npar, cols = nd.cols;
    const float* __restrict__ Vhi = ws + nd.v_off;
    const float* __restrict__ Vlo = ws + nd.v_off + R * cols;
    float* myU = sU + warp * kTile;
    const int nw = min(S, kWarps);
    // V_r staging: thread -> 4 entries (row e / 32, column lane) of the 32 x 32 tile;
    // the next rep's values are loaded into registers while this rep computes
    float vn[4];
    auto load_v = [&](int r) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + q * kThreads, row = e >> 5, col = e & 31;
            vn[q] = 0.f;
            if (r < it.a + it.b && row < n_j1 && col < n_j2) {
                const int64_t o = (int64_t)r * cols + (int64_t)row * n_j2 + col;
                vn[q] = Vhi[o] + Vlo[o];
            }
        }
    };
    auto store_v = [&](float* dst) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + q * kThreads;
            dst[swz(e >> 5, e & 31)] = vn[q];
        }
    };
    load_v(it.a);
    store_v(sV);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // this thread's A / B copies (the loop's barrier publishes all)
    for (int r = it.a; r < it.a + it.b; ++r) {
        float* cur = sV + ((r - it.a) & 1) * kTile;
        __syncthreads();  // A, B and this rep's V staged; the previous rep's reduction has read sU
        load_v(r + 1);
        float w[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) w[i][j] = 0.f;
        for (int s = warp; s < S; s += kWarps) {
            float u[4][8];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) u[i][j] = 0.f;
            tile_nt(sB + s * kTile, cur, ab, bb, u);  // U_s[i2][j1]
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) myU[swz(ab + 8 * i, bb + 4 * j)] = u[i][j];
            __syncwarp();
            tile_nt(sA + s * kTile, myU, ab, bb, w);  // W[i1][i2] += A_s U_s^T
            __syncwarp();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) myU[swz(ab + 8 * i, bb + 4 * j)] = w[i][j];
        store_v(sV + ((r + 1 - it.a) & 1) * kTile);  // the other buffer: no one reads it now
        __syncthreads();
        // sum of the warps' partial tiles: thread -> row i1 = tid / 8, columns 4 (tid % 8) ..
        const int row = tid >> 3, c4 = tid & 7;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int q = 0; q < nw; ++q) {
            const float4 x = *reinterpret_cast<const float4*>(sU + q * kTile + row * 32 + ((c4 ^ (row & 7)) << 2));
            acc.x += x.x;
            acc.y += x.y;
            acc.z += x.z;
            acc.w += x.w;
        }
        if (row < n_i1) {
            float* dst = ws + nd.w_off + (int64_t)r * npar + (int64_t)row * n_i2 + 4 * c4;
            if (n_i2 == 32 && ((uintptr_t)dst & 15) == 0) {
                *reinterpret_cast<float4*>(dst) = acc;
            } else {
                const float a4[4] = {acc.x, acc.y, acc.z, acc.w};
                for (int q = 0; q < 4; ++q)
                    if (4 * c4 + q < n_i2) dst[q] = a4[q];
            }
        }
    }
}

size_t m2_rung_fact_smem(int s) { return (size_t)(2 * s + 2 + kWarps) * kTile * sizeof(float); }

cudaError_t launch_m2_rung_fact(int n, const M2Node* nodes, const M2Net* nets, const M2Item* items, float* ws,
                                size_t smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(m2_rung_fact_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    m2_rung_fact_kernel<<<n, kThreads, smem, s>>>(nodes, nets, items, ws);
    return cudaGetLastError();
}

}  // namespace tnsk
