// m2_rung_tc.cu -- method 2's sketched product (row a7, Alg. 5) for a grouped tensor
// in factored form on the 5th-generation tensor cores.
//
// A grouped (rung) tensor is X((i1,i2),(j1,j2)) = sum_s A(i1,s,j1) B(i2,s,j2): the
// exact grouping of Sec. 4.1, indices named by the node's row / column split. The
// product W^T[r][(i1,i2)] = sum_{j1,j2} X((i1,i2),(j1,j2)) V[r][(j1,j2)] is taken
// in two contractions, so X's entries are never formed (2 s n^3 multiply-adds per
// rep for n = 32 instead of the n^4 of the dense product; only A and B are read):
//   U[(r,j1),(s,i2)] = sum_{j2} V[r][(j1,j2)] B(i2,s,j2)     (step 1)
//   W[(r,i2), i1]    = sum_{s,j1} U[(r,j1),(s,i2)] A(i1,s,j1)  (step 2)
// Both are tcgen05.mma products (kind::tf32, FP32 accumulators in tensor memory,
// every operand split as hi + lo TF32 parts and the three products hi.hi + hi.lo +
// lo.hi summed, as in the streaming kernel). All four factor dims are 32 and
// s <= 8; a block of 4 reps makes the 128 tensor-memory lanes (r, j1) of step 1
// and (r, i2) of step 2.
//
// Step 1 reads V^T as stored by the V build ([R][(j1,j2)], viewed as [(r,j1)][j2]:
// 128-byte rows) by TMA, and B as [(s,i2)][j2] from a prepared copy. Its result
// U sits in tensor memory with lanes (r, j1); step 2 needs lanes (r, i2) with K =
// j1, so the converter warps read U one s at a time (32 columns), transpose the
// 32 x 32 block of their rep through shared memory, split it into TF32 hi / lo and
// store it back to tensor memory as step 2's A operand; B of step 2 is A(i1,s,j1)
// as [s][i1][j1] from the prepared copy.
//
// m2_rung_prep_kernel writes the prepared copy once per run: per node the hi and lo
// parts of B as [(s,i2)][j2] and of A as [(s,i1)][j1], each a 128-byte-row image of
// the 128-byte-swizzled K-major layout, so that one plain bulk copy per part lands
// it in shared memory ready for the tensor core.
#include <algorithm>

#include "common.cuh"
#include "method2.cuh"
#include "tcgen05.cuh"

namespace tnsk {

// Byte offset of (row, k) (k < 32) in a K-major FP32 tile with 128-byte rows and the
// 128-byte swizzle: 16-byte chunk k / 4 of a row goes to chunk (k / 4) xor (row % 8).
__host__ __device__ __forceinline__ int sw128_offset(int row, int k) {
    return row * 128 + ((((k >> 2) ^ (row & 7))) << 4) + (k & 3) * 4;
}

// One block per grouped node: the hi / lo TF32 parts of B(i2,s,j2) at row s 32 + i2,
// column j2 and of A(i1,s,j1) at row s 32 + i1, column j1 (parts [Bh | Bl | Ah | Al],
// each s 4 KiB), split exactly as the streaming kernel splits its operands. A thread
// writes one 16-byte chunk (4 columns) of a row in each part.
__global__ void __launch_bounds__(256) m2_rung_prep_kernel(const M2Node* __restrict__ nodes,
                                                           const M2Item* __restrict__ items, float* __restrict__ ws) {
    const M2Node& nd = nodes[items[blockIdx.x].node];
    const int S = nd.rs;
    const size_t part = (size_t)S * 4096;  // bytes per part
    unsigned char* dst = reinterpret_cast<unsigned char*>(ws + nd.rc_off);
    const float* __restrict__ gA = nd.rA;
    const float* __restrict__ gB = nd.rB;
    for (int e = threadIdx.x; e < S * 32 * 8; e += blockDim.x) {
        const int row = e >> 3, c = e & 7;  // row s 32 + x, columns 4 c .. 4 c + 3
        const int s = row >> 5, x = row & 31;
        uint32_t bh[4], bl[4], ah[4], al[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int k = 4 * c + u;
            tf32_split(__ldg(gB + (int64_t)x * nd.r_bi + (int64_t)k * nd.r_bj + (int64_t)s * nd.r_bs), bh[u], bl[u]);
            tf32_split(__ldg(gA + (int64_t)x * nd.r_ai + (int64_t)k * nd.r_aj + (int64_t)s * nd.r_as), ah[u], al[u]);
        }
        const size_t off = (size_t)sw128_offset(row, 4 * c);
        *reinterpret_cast<uint4*>(dst + off) = make_uint4(bh[0], bh[1], bh[2], bh[3]);
        *reinterpret_cast<uint4*>(dst + part + off) = make_uint4(bl[0], bl[1], bl[2], bl[3]);
        *reinterpret_cast<uint4*>(dst + 2 * part + off) = make_uint4(ah[0], ah[1], ah[2], ah[3]);
        *reinterpret_cast<uint4*>(dst + 3 * part + off) = make_uint4(al[0], al[1], al[2], al[3]);
    }
}

cudaError_t launch_m2_rung_prep(int n, const M2Node* nodes, const M2Item* items, float* ws, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    m2_rung_prep_kernel<<<n, 256, 0, s>>>(nodes, items, ws);
    return cudaGetLastError();
}

namespace {

constexpr int kRtReps = 4;             // reps per block: 4 x 32 = 128 tensor-memory lanes
static_assert(kRtReps * 32 == 128, "a block's reps fill the 128 lanes");
constexpr int kRtThreads = 320;        // warp 0 loads, warp 1 MMA, warps 2-9 converters
constexpr int kRtPart = 32 * 1024;     // shared bytes of one prepared part (s <= 8)
constexpr int kRtV = 128 * 128;        // one of V^T hi / lo for a block: 128 rows x 128 B
constexpr int kRtScratch = 32 * 33 * 4;  // per converter warp: a 32 x 32 FP32 block, rows padded to 33
// shared memory: [Bh | Bl | Ah | Al] (4 x 32 KiB), V^T ring (2 stages x hi + lo),
// transpose scratch (8 warps), + alignment slack
constexpr int kRtSmem = 4 * kRtPart + 2 * 2 * kRtV + 8 * kRtScratch + 1024;
// with the static part (barriers, the block table: under 1 KiB) within the 227 KiB a CTA may use
static_assert(kRtSmem <= 227 * 1024 - 1024, "shared memory of m2_rung_tc_kernel");
// tensor memory (512 columns): U's halves at [0, 32 S0) and [128, 128 + 32 (s - S0)) with
// S0 = ceil(s / 2); step 2's A stages at 256 + 64 t (hi in the first 32 columns, lo in the
// next 32); W as four partial sums at 384 + 32 a (a = the K step of 8 within each s: the
// MMAs into different sums do not wait for one another)
constexpr uint32_t kRtCols = 512;
constexpr uint32_t kRtA2 = 256;
constexpr uint32_t kRtW = 384;

// Instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t rt_idesc(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void rt_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar)));
}

// One block of the CTA's range, read once at the start (the roles' loops then read
// shared memory, not the descriptors in global memory).
struct RtBlk {
    int32_t node, r0, nrep, S;    // node, first rep, reps (<= 4), s
    int32_t first, last;          // first / last block of its node in this CTA
    int32_t tm_v;                 // tensor maps of V^T hi / lo (tm_v, tm_v + 1)
    int32_t npar;                 // W^T row length
    int64_t rc_off, w_off;        // prepared factors, W^T
};
constexpr int kRtMaxBlk = 16;  // blocks per CTA per launch (the launcher splits larger lists)
}  // namespace

// Persistent: CTA g takes the blocks (node, 4 reps) items[g n / G .. (g + 1) n / G) in
// order (node-major), reloading the prepared factors when the node changes. The MMA
// thread interleaves the next block's step 1 with this block's step 2 (half of U's
// columns at a time), so that the tensor core works while the converters transpose:
//   step1(0, h0) step1(0, h1) | per block q: step2(q, s in h0) step1(q+1, h0)
//                               step2(q, s in h1) step1(q+1, h1)
// The converters are two groups of four warps (one warp per lane quarter each) that
// take the s values of a block in turn, group g always filling step 2's A stage g.
// Barriers: factor parts (full: TMA bytes; empty: the MMAs reading them done), V^T
// stages (same), U halves (full: step 1 done; empty: all eight converter warps have
// read it), step 2's A stages (full: the group's stores; empty: the MMAs done), W
// (full: step 2 of the block done; empty: both groups' epilogues have read it).
__global__ void __launch_bounds__(kRtThreads, 1) m2_rung_tc_kernel(const M2Node* __restrict__ nodes,
                                                                   const M2Item* __restrict__ items, int n_items,
                                                                   float* __restrict__ ws,
                                                                   const unsigned char* __restrict__ tmaps,
                                                                   int* __restrict__ err, int inject) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t b_full, b_empty, a_full, a_empty;
    __shared__ __align__(8) uint64_t v_full[2], v_empty[2];
    __shared__ __align__(8) uint64_t y_full[2], y_empty[2];
    __shared__ __align__(8) uint64_t a2_full[2], a2_empty[2];
    __shared__ __align__(8) uint64_t d_full, w_empty;
    __shared__ uint32_t tmem_base;
    __shared__ RtBlk blk[kRtMaxBlk];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sBh = sm;
    unsigned char* sBl = sm + kRtPart;
    unsigned char* sAh = sm + 2 * kRtPart;
    unsigned char* sAl = sm + 3 * kRtPart;
    unsigned char* sV = sm + 4 * kRtPart;  // stage t: hi at t 2 kRtV, lo kRtV after it
    float* sT = reinterpret_cast<float*>(sV + 4 * kRtV);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x;
    const int beg = (int)(((int64_t)n_items * blockIdx.x) / G);
    const int nb = min((int)(((int64_t)n_items * (blockIdx.x + 1)) / G) - beg, kRtMaxBlk);

    for (int q = tid; q < nb; q += kRtThreads) {
        const M2Item it = items[beg + q];
        const M2Node& nd = nodes[it.node];
        RtBlk b;
        b.node = it.node;
        b.r0 = it.a;
        b.nrep = it.b;
        b.S = nd.rs;
        b.first = q == 0 || items[beg + q - 1].node != it.node;
        b.last = q == nb - 1 || items[beg + q + 1].node != it.node;
        b.tm_v = nd.tm_v;
        b.npar = (int32_t)nd.npar;
        b.rc_off = nd.rc_off;
        b.w_off = nd.w_off;
        blk[q] = b;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(kRtCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        auto init = [](uint64_t* b, uint32_t n) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(n));
        };
        init(&b_full, 1);
        init(&b_empty, 1);
        init(&a_full, 1);
        init(&a_empty, 1);
        init(&d_full, 1);
        for (int t = 0; t < 2; ++t) {
            init(&v_full[t], 1);
            init(&v_empty[t], 1);
            init(&y_full[t], 1);
            init(&a2_empty[t], 1);
            init(&a2_full[t], 4);  // the four warps of group t
            init(&y_empty[t], 8);  // all eight converter warps
        }
        init(&w_empty, 8);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    bool ok = true;

    if (warp == 0) {
        // ---------------- loads (one thread): per block its V^T tiles; per node change the
        // prepared factors, B once step 1 of the previous node is done, A once its step 2
        // is. With a test's injected fault nothing is loaded (the consumers' bounded waits
        // run out). Before leaving it waits (bounded) for its last loads to land.
        if (lane == 0 && !inject && nb > 0) {
            int loads = 0;
            for (int q = 0; q < nb && ok; ++q) {
                const RtBlk& b = blk[q];
                const int vs = q & 1;
                if (q >= 2) ok = mbar_wait(smem_addr(&v_empty[vs]), (uint32_t)(((q >> 1) - 1) & 1));
                if (!ok) break;
                const void* tmvh = tmaps + (int64_t)b.tm_v * 128;
                const void* tmvl = tmaps + (int64_t)(b.tm_v + 1) * 128;
                if (b.first) {
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmvh) : "memory");
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmvl) : "memory");
                }
                const uint32_t vb = smem_addr(&v_full[vs]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(vb), "r"(2 * kRtV)
                             : "memory");
                tma_load_2d(smem_addr(sV + vs * 2 * kRtV), tmvh, 0, b.r0 * 32, vb);
                tma_load_2d(smem_addr(sV + vs * 2 * kRtV + kRtV), tmvl, 0, b.r0 * 32, vb);
                if (b.first) {
                    const uint32_t bytes = (uint32_t)b.S * 4096u;
                    const unsigned char* src = reinterpret_cast<const unsigned char*>(ws + b.rc_off);
                    if (loads >= 1) ok = mbar_wait(smem_addr(&b_empty), (uint32_t)((loads - 1) & 1));
                    if (!ok) break;
                    const uint32_t bb = smem_addr(&b_full);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bb), "r"(2 * bytes)
                                 : "memory");
                    bulk_load(smem_addr(sBh), src, bytes, bb);
                    bulk_load(smem_addr(sBl), src + bytes, bytes, bb);
                    if (loads >= 1) ok = mbar_wait(smem_addr(&a_empty), (uint32_t)((loads - 1) & 1));
                    if (!ok) break;
                    const uint32_t ab = smem_addr(&a_full);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ab), "r"(2 * bytes)
                                 : "memory");
                    bulk_load(smem_addr(sAh), src + 2 * bytes, bytes, ab);
                    bulk_load(smem_addr(sAl), src + 3 * bytes, bytes, ab);
                    ++loads;
                }
            }
            // the last loads in flight: the last two V^T stages and the last factors
            for (int q = nb >= 2 ? nb - 2 : 0; q < nb; ++q)
                if (!mbar_wait(smem_addr(&v_full[q & 1]), (uint32_t)((q >> 1) & 1))) ok = false;
            if (loads >= 1) {
                if (!mbar_wait(smem_addr(&b_full), (uint32_t)((loads - 1) & 1))) ok = false;
                if (!mbar_wait(smem_addr(&a_full), (uint32_t)((loads - 1) & 1))) ok = false;
            }
        }
        __syncwarp();
    }
    else if (warp == 1) {
        // ---------------- MMA issue (one thread)
        if (lane == 0 && nb > 0) {
            int bl = 0, al = 0, c2 = 0;
            int yuse0 = 0, yuse1 = 0;  // uses of U's halves (scalars: no local-memory array)
            // step 1 of block q, half h of U (s in [h S0, h S0 + nh)) into columns h 128 ..:
            // fixed places, so that blocks of nodes with different s never overlap halves
            auto step1 = [&](int q, int h) {
                const RtBlk& b = blk[q];
                const int S = b.S, S0 = (S + 1) >> 1;
                const int nh = h ? S - S0 : S0;
                if (nh == 0 || !ok) return;
                if (h == 0) {
                    if (b.first) ok = mbar_wait(smem_addr(&b_full), (uint32_t)(bl++ & 1));
                    ok = ok && mbar_wait(smem_addr(&v_full[q & 1]), (uint32_t)((q >> 1) & 1));
                }
                const int yu = h ? yuse1++ : yuse0++;
                if (yu >= 1) ok = ok && mbar_wait(smem_addr(&y_empty[h]), (uint32_t)((yu - 1) & 1));
                if (!ok) return;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t vst = smem_addr(sV + (q & 1) * 2 * kRtV);
                const uint32_t brow = (uint32_t)(h * S0 * 32 * 128);
                const uint32_t aop[3] = {vst, vst, vst + kRtV};  // V hi.B hi + V hi.B lo + V lo.B hi
                const uint32_t bop[3] = {smem_addr(sBh) + brow, smem_addr(sBl) + brow, smem_addr(sBh) + brow};
                const uint32_t idesc = rt_idesc(nh * 32);
                const uint32_t d = tmem + (uint32_t)(h * 128);
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t ad = smem_desc_sw128(aop[p] + ks * 32);
                        const uint64_t bd = smem_desc_sw128(bop[p] + ks * 32);
                        const uint32_t acc = (p > 0 || ks > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n\t}" ::"r"(d),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                    }
                rt_commit(&y_full[h]);
                if (h == 1 || S0 == S) {  // the block's last step-1 MMAs: its V^T stage is free
                    rt_commit(&v_empty[q & 1]);
                    if (b.last) rt_commit(&b_empty);
                }
            };
            // step 2 of block q for one s: W += U_s^T A_s^T over K = j1
            auto step2 = [&](int q, int s) {
                const RtBlk& b = blk[q];
                if (!ok) return;
                if (s == 0 && b.first) ok = mbar_wait(smem_addr(&a_full), (uint32_t)(al++ & 1));
                if (s == 0 && q >= 1) ok = ok && mbar_wait(smem_addr(&w_empty), (uint32_t)((q - 1) & 1));
                const int t = c2 & 1;
                ok = ok && mbar_wait(smem_addr(&a2_full[t]), (uint32_t)((c2 >> 1) & 1));
                ++c2;
                if (!ok) return;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ahi = tmem + kRtA2 + 64u * (uint32_t)t, alo = ahi + 32;
                const uint32_t aop[3] = {ahi, ahi, alo};
                const uint32_t bo = (uint32_t)s * 4096u;
                const uint32_t bop[3] = {smem_addr(sAh) + bo, smem_addr(sAl) + bo, smem_addr(sAh) + bo};
                const uint32_t idesc = rt_idesc(32);
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t bd = smem_desc_sw128(bop[p] + ks * 32);
                        const uint32_t acc = (s > 0 || p > 0) ? 1u : 0u;  // partial sum ks
                        asm volatile(
                            "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, q;\n\t}" ::"r"(tmem + kRtW + 32u * (uint32_t)ks),
                            "r"(aop[p] + ks * 8), "l"(bd), "r"(idesc), "r"(acc));
                    }
                rt_commit(&a2_empty[t]);
                if (s == b.S - 1) {
                    rt_commit(&d_full);
                    if (b.last) rt_commit(&a_empty);
                }
            };
            step1(0, 0);
            step1(0, 1);
            for (int q = 0; q < nb && ok; ++q) {
                const int S = blk[q].S, S0 = (S + 1) >> 1;
                for (int s = 0; s < S0; ++s) step2(q, s);
                if (q + 1 < nb) step1(q + 1, 0);
                for (int s = S0; s < S; ++s) step2(q, s);
                if (q + 1 < nb) step1(q + 1, 1);
            }
        }
        __syncwarp();
    }
    else {
        // ---------------- converters (warps 2-9): warp w serves tensor-memory lanes
        // 32 (w % 4) .. + 31, rep rr = w % 4 of each block; group g = (w - 2) / 4 takes the
        // block's s values whose running index c2 has parity g. Lane = j1 when reading U,
        // i2 when writing step 2's operand.
        const int rr = warp & 3, g = (warp - 2) >> 2;
        const uint32_t lane_base = (uint32_t)(rr * 32) << 16;
        float* T = sT + (warp - 2) * 32 * 33;  // element (row, col) at row 33 + col
        int c2 = 0;
        int yuse0 = 0, yuse1 = 0;
        for (int q = 0; q < nb && ok; ++q) {
            const RtBlk& b = blk[q];
            const int S = b.S, S0 = (S + 1) >> 1;
            for (int h = 0; h < 2 && ok; ++h) {
                const int nh = h ? S - S0 : S0;
                if (nh == 0) continue;
                const int yu = h ? yuse1++ : yuse0++;
                ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&y_full[h]), (uint32_t)(yu & 1)));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // this group's last s of the half (-1: none): after reading it, U's half is
                // released by this warp
                int jl = -1;
                for (int j = 0; j < nh; ++j)
                    if (((c2 + j) & 1) == g) jl = j;
                if (jl < 0 && lane == 0) mbar_arrive(smem_addr(&y_empty[h]));
                for (int j = 0; j < nh; ++j, ++c2) {
                    if ((c2 & 1) != g) continue;
                    uint32_t v[32];
                    tmem_load32(tmem + lane_base + (uint32_t)(h * 128 + j * 32), v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (j == jl) {
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) mbar_arrive(smem_addr(&y_empty[h]));
                    }
                    // the rep's 32 x 32 block transposed: v[i2] of lane j1 -> column j1 of lane i2
#pragma unroll
                    for (int i2 = 0; i2 < 32; ++i2) T[i2 * 33 + lane] = __uint_as_float(v[i2]);
                    __syncwarp();
                    // split into TF32 hi / lo and stored 16 columns at a time (fewer live
                    // registers); the A stage is waited for between the two halves
                    const uint32_t col = kRtA2 + 64u * (uint32_t)g;
#pragma unroll
                    for (int part = 0; part < 2; ++part) {
                        uint32_t hi[16], lo[16];
#pragma unroll
                        for (int j1 = 0; j1 < 16; ++j1)
                            tf32_split(T[lane * 33 + 16 * part + j1], hi[j1], lo[j1]);
                        if (part == 0) {
                            bool w_ok = true;
                            if (c2 >= 2) w_ok = mbar_wait(smem_addr(&a2_empty[g]), (uint32_t)(((c2 >> 1) - 1) & 1));
                            ok = __all_sync(0xffffffffu, w_ok);
                            if (!ok) break;
                        }
                        tmem_store16(tmem + lane_base + col + 16u * (uint32_t)part, hi);
                        tmem_store16(tmem + lane_base + col + 32u + 16u * (uint32_t)part, lo);
                    }
                    __syncwarp();  // every lane's reads of T done before the next s overwrites it
                    if (!ok) break;
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_addr(&a2_full[g]));
                }
            }
            if (!ok) break;
            // ---------------- epilogue: W_r[i1][i2] for r = r0 + rr, i2 = lane, i1 in
            // [16 g, 16 g + 16): the four partial sums added, stored as W^T rows
            ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&d_full), (uint32_t)(q & 1)));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float acc[16];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                uint32_t w[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]),
                      "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]),
                      "=r"(w[15])
                    : "r"(tmem + lane_base + kRtW + 32u * (uint32_t)a + 16u * (uint32_t)g));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[i] = a == 0 ? __uint_as_float(w[i]) : acc[i] + __uint_as_float(w[i]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&w_empty));  // the next block's step 2 may overwrite W
            if (rr < b.nrep) {
                float* dst = ws + b.w_off + (int64_t)(b.r0 + rr) * b.npar + 16 * g * 32 + lane;
#pragma unroll
                for (int i = 0; i < 16; ++i) dst[i * 32] = acc[i];
            }
        }
    }
    if (!ok && lane == 0) atomicExch(err, DEVERR_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kRtCols));
}

cudaError_t launch_m2_rung_tc(int n, const M2Node* nodes, const M2Item* items, float* ws, const unsigned char* tmaps,
                              int* err, int inject, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    static int sms = 0;  // one persistent CTA per SM (the kernel's shared memory allows one)
    if (sms <= 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    }
    cudaError_t e = cudaFuncSetAttribute(m2_rung_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kRtSmem);
    if (e != cudaSuccess) return e;
    // at most kRtMaxBlk blocks per CTA: longer lists in several launches
    const int chunk = kRtMaxBlk * sms;
    for (int off = 0; off < n; off += chunk) {
        const int cnt = std::min(chunk, n - off);
        m2_rung_tc_kernel<<<std::min(cnt, sms), kRtThreads, kRtSmem, s>>>(nodes, items + off, cnt, ws, tmaps, err,
                                                                            inject);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace tnsk
