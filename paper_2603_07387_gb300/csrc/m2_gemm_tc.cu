// m2_gemm_tc.cu -- row a7 of the hot path on the 5th-generation tensor cores.
//
// The sketched matrix-vector product of Alg. 5, for all repetitions at once,
// is the dense product W = mat(X_k) V (V(col, r) = sigma_r(col) r_k[r][b_r(col)])
// followed by the count-sketch scatter of W's rows into x_k. This kernel computes
// a 128-row x 64-rep tile of W with tcgen05.mma (kind::tf32, FP32 accumulators in
// tensor memory) and writes it as W^T (coalesced rows); m2_wscatter_kernel then
// applies the count sketch of the parent edge with shared-memory bins.
//
// FP32 accuracy from TF32 tensor cores: every operand value v is split as
// v = hi + lo with hi = tf32(v) (round to nearest) and lo = tf32(v - hi), and
// W = Xhi Vhi + Xhi Vlo + Xlo Vhi (the dropped Xlo Vlo is below 2^-22 relative).
//
// General kernel (any dtype, any parent mode, any column count): per K-chunk of
// 32 columns, X (128 x 32) and V^T (64 x 32) tiles are staged in shared memory
// in the K-major, no-swizzle canonical layout: core matrices of 8 rows x 16
// bytes; K-adjacent cores 128 B apart (leading byte offset), 8-row groups 1024 B
// apart (stride byte offset). Two stages: threads load chunk c+1 into registers
// while the tensor core works on chunk c; an mbarrier signalled by tcgen05.commit
// frees a stage. The streaming kernel further below serves the common case.
#include "common.cuh"
#include "method2.cuh"
#include "tcgen05.cuh"

namespace tnsk {
namespace {

constexpr int kTM = 128;  // rows of W per CTA (TMEM lanes)
constexpr int kTN = 64;   // reps per CTA (TMEM columns)
constexpr int kKC = 32;   // columns per chunk (4 MMAs of K = 8)
constexpr int kStages = 2;
constexpr int kABytes = kTM * kKC * 4;                   // 16 KiB
constexpr int kBBytes = kTN * kKC * 4;                   // 8 KiB
constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes;   // hi + lo of both
constexpr int kSmemBytes = kStages * kStageBytes + 1024;  // + alignment slack

// Byte offset of (row, k) in a K-major no-swizzle operand tile (k < 32).
__device__ __forceinline__ int kmajor_offset(int row, int k) {
    return (row >> 3) * 1024 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// Shared-memory matrix descriptor: start, leading / stride byte offsets (>> 4),
// descriptor version 1 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, N = 64, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ void store_split(unsigned char* hi, unsigned char* lo, int off, float4 v) {
    uint32_t h0, h1, h2, h3, l0, l1, l2, l3;
    tf32_split(v.x, h0, l0);
    tf32_split(v.y, h1, l1);
    tf32_split(v.z, h2, l2);
    tf32_split(v.w, h3, l3);
    *reinterpret_cast<uint4*>(hi + off) = make_uint4(h0, h1, h2, h3);
    *reinterpret_cast<uint4*>(lo + off) = make_uint4(l0, l1, l2, l3);
}

}  // namespace

// One CTA (128 threads) per item: (node, 128-row tile it.a, 64-rep tile it.b, K split
// it.pad_ of it.begin).
__global__ void __launch_bounds__(128, 2) m2_gemm_tc_kernel(const M2Node* __restrict__ nodes,
                                                            const M2Net* __restrict__ nets,
                                                            const M2Item* __restrict__ items,
                                                            const uint32_t* __restrict__ tabs, float* __restrict__ ws,
                                                            int* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t empty_bar[kStages];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_base;
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const M2Item it = items[blockIdx.x];
    const M2Node& nd = nodes[it.node];
    const M2Net& N = nets[nd.net];
    const int R = N.R;
    const int64_t row0 = (int64_t)it.a * kTM;
    const int rep0 = it.b * kTN;
    const int64_t npar = nd.npar, cols = nd.cols, Bc = nd.Bc;
    const float* V = ws + nd.v_off;                       // TF32 hi part of V^T
    const float* Vlo = ws + nd.v_off + (int64_t)R * cols;  // its lo part
    const bool fast_x = nd.dtype == TNSK_F32 && nd.A == 1 && (cols & 3) == 0 &&
                        ((uintptr_t)nd.data & 15) == 0;
    const bool fast_v = (cols & 3) == 0 && (((uintptr_t)V) & 15) == 0 && (((uintptr_t)Vlo) & 15) == 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(kTN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&empty_bar[s])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&done_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    // thread -> 16-byte column group `sub` of rows rin + 8 (rhi + 2 j): the 8 threads of a
    // quarter warp share a column group and cover the 8 rows of a core matrix, so
    // their 16-byte stores land in 8 different bank groups
    const int rin = tid & 7, sub = (tid >> 3) & 7, rhi = tid >> 6;
    auto trow = [&](int j) { return rin + 8 * (rhi + 2 * j); };
    float4 ra[8], rv[4], rvl[4];
    auto load_chunk = [&](int64_t k0) {
        const int64_t gc = k0 + sub * 4;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t gr = row0 + trow(j);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gr < npar) {
                if (fast_x) {
                    if (gc < cols) v = __ldg(reinterpret_cast<const float4*>((const float*)nd.data + gr * Bc + gc));
                } else {
                    float t[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int64_t cc = gc + q;
                        t[q] = 0.f;
                        if (cc < cols) {
                            const int64_t a = cc / Bc;
                            t[q] = load_as<float>(nd.data, nd.dtype, (a * npar + gr) * Bc + (cc - a * Bc));
                        }
                    }
                    v = make_float4(t[0], t[1], t[2], t[3]);
                }
            }
            ra[j] = v;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int rep = rep0 + trow(j);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f), vl = v;
            if (rep < R) {
                const float* src = V + (int64_t)rep * cols;
                const float* srl = Vlo + (int64_t)rep * cols;
                if (fast_v) {
                    if (gc < cols) {
                        v = *reinterpret_cast<const float4*>(src + gc);
                        vl = *reinterpret_cast<const float4*>(srl + gc);
                    }
                } else {
                    v.x = gc + 0 < cols ? src[gc + 0] : 0.f;
                    v.y = gc + 1 < cols ? src[gc + 1] : 0.f;
                    v.z = gc + 2 < cols ? src[gc + 2] : 0.f;
                    v.w = gc + 3 < cols ? src[gc + 3] : 0.f;
                    vl.x = gc + 0 < cols ? srl[gc + 0] : 0.f;
                    vl.y = gc + 1 < cols ? srl[gc + 1] : 0.f;
                    vl.z = gc + 2 < cols ? srl[gc + 2] : 0.f;
                    vl.w = gc + 3 < cols ? srl[gc + 3] : 0.f;
                }
            }
            rv[j] = v;
            rvl[j] = vl;
        }
    };

    // this item's share of the K chunks (split K: partial tiles meet in the atomic scatter)
    const int total_chunks = (int)((cols + kKC - 1) / kKC);
    const int cbeg = (int)(((int64_t)total_chunks * it.pad_) / it.begin);
    const int cend = (int)(((int64_t)total_chunks * (it.pad_ + 1)) / it.begin);
    const int nchunks = cend - cbeg;
    bool ok = true;
    if (nchunks > 0) load_chunk((int64_t)cbeg * kKC);
    for (int c = 0; c < nchunks; ++c) {
        const int s = c % kStages;
        unsigned char* st = sm + s * kStageBytes;
        unsigned char *a_hi = st, *a_lo = st + kABytes, *b_hi = st + 2 * kABytes, *b_lo = st + 2 * kABytes + kBBytes;
        if (c >= kStages) ok = mbar_wait(smem_addr(&empty_bar[s]), (uint32_t)((c / kStages - 1) & 1)) && ok;
#pragma unroll
        for (int j = 0; j < 8; ++j) store_split(a_hi, a_lo, kmajor_offset(trow(j), sub * 4), ra[j]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int off = kmajor_offset(trow(j), sub * 4);
            *reinterpret_cast<float4*>(b_hi + off) = rv[j];
            *reinterpret_cast<float4*>(b_lo + off) = rvl[j];
        }
        if (c + 1 < nchunks) load_chunk((int64_t)(cbeg + c + 1) * kKC);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned char* aop[3] = {a_hi, a_hi, a_lo};
            const unsigned char* bop[3] = {b_hi, b_lo, b_hi};
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int ks = 0; ks < kKC / 8; ++ks) {
                    const uint64_t ad = smem_desc(smem_addr(aop[p]) + ks * 256, 128, 1024);
                    const uint64_t bd = smem_desc(smem_addr(bop[p]) + ks * 256, 128, 1024);
                    const uint32_t acc = (c > 0 || p > 0 || ks > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n\t}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&empty_bar[s])));
            if (c == nchunks - 1)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(&done_bar)));
        }
    }
    if (nchunks > 0) ok = mbar_wait(smem_addr(&done_bar), 0u) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if (lane == 0) atomicExch(err, DEVERR_TIMEOUT);
    } else if (nchunks > 0) {
        // epilogue: row = this thread's TMEM lane; x_k[r][h(row)] += s(row) W[row][r]
        const int64_t row = row0 + warp * 32 + lane;
#pragma unroll
        for (int cc = 0; cc < kTN / 16; ++cc) {
            uint32_t v[16];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 16);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < npar) {
                // W^T[rep][row]: a warp writes 32 consecutive rows of one rep
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int rep = rep0 + cc * 16 + j;
                    if (rep < R) {
                        float* dst = &ws[nd.w_off + (int64_t)rep * npar + row];
                        if (it.begin > 1)
                            atomicAdd(dst, __uint_as_float(v[j]));  // K split: partial sums
                        else
                            *dst = __uint_as_float(v[j]);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTN));
}

// ---------------------------------------------------------------------------
// Streaming variant for row-major FP32 tensors whose parent mode is the first
// mode (mat(X_k) is the row-major matrix itself) and whose column count is a
// multiple of 4. Warp-specialised; per K-chunk of 32 columns the tile of X and the
// tiles of the pre-split V^T (hi and lo TF32 parts, written by the V build) arrive
// by TMA (2-D boxes from tensor maps made at plan time) in the 128-byte swizzled
// K-major layout, with zero fill outside the matrices. X's hi / lo parts go to
// tensor memory, so the MMA reads A from TMEM and only B from shared memory. X and
// V^T have rings of their own (3 deep each): an X stage is free again as soon as the
// converters have read it, a V^T stage once the MMA that reads it completes; three
// TMEM operand stages let the conversion of a chunk overlap the MMAs of the two
// before it. X loads are marked evict-first in L2, V^T loads evict-last:
//   warp 0     X producer: one cp.async.bulk.tensor load per chunk
//   warps 1-4  converters: one row of X per thread (its TMEM lane), raw FP32 ->
//              hi / lo TF32 stored with tcgen05.st; then the epilogue
//   warp 5     tensor memory allocation and MMA issue: one wait (tm_full: the
//              converters' TMEM stores, and the V^T tiles, checked by one converter) and
//              one tcgen05.commit (freeing the V^T stage and the TMEM stage) per chunk
//   warp 6     V^T producer: the hi and lo tiles of each chunk (L2-resident: the
//              row tiles of one matrix share them)
// Two CTAs share an SM, so one's prologue and epilogue overlap the other's streaming.
// Tensor memory: columns [0, 64) accumulator, [64 + 64 t, + 64) operand stage t
// (hi in the first 32 columns, lo in the next 32).
// ---------------------------------------------------------------------------
namespace {

constexpr int kXStages = 3;    // X ring; two CTAs per SM: 2 x 97 KiB of shared memory
constexpr int kVStages = 3;    // V^T ring
constexpr int kTmStages = 3;   // TMEM operand stages: columns 64 + 64 t, t < 3, of 256
static_assert(kVStages == kTmStages, "chunk c uses V^T stage and TMEM stage c % 3: one barrier frees both");
constexpr int kRawX = kTM * 128;   // 128 rows x 128 B
constexpr int kRawV = kTN * 128;   // 64 rows x 128 B (one of hi / lo)
constexpr int kStreamThreads = 224;
constexpr int kStreamSmem = kXStages * kRawX + kVStages * 2 * kRawV + 1024;
constexpr uint32_t kTmemCols = 256;

}  // namespace

__global__ void __launch_bounds__(kStreamThreads, 2) m2_gemm_tc_stream_kernel(const M2Node* __restrict__ nodes,
                                                                               const M2Net* __restrict__ nets,
                                                                               const M2Item* __restrict__ items,
                                                                               float* __restrict__ ws,
                                                                               const unsigned char* __restrict__ tmaps,
                                                                               int* __restrict__ err, int inject) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t x_full[kXStages], x_empty[kXStages];
    __shared__ __align__(8) uint64_t v_full[kVStages];
    // tm_full[t]: TMEM operand stage t written and V^T stage t landed (one wait for the
    // MMA thread); freed[t]: the MMAs of stage t done (one commit frees both stages)
    __shared__ __align__(8) uint64_t tm_full[kTmStages], freed[kTmStages];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_base;
    unsigned char* xring = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* vring = xring + kXStages * kRawX;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const M2Item it = items[blockIdx.x];
    const M2Node& nd = nodes[it.node];
    const M2Net& N = nets[nd.net];
    const int R = N.R;
    const int64_t row0 = (int64_t)it.a * kTM;
    const int rep0 = it.b * kTN;
    const int64_t npar = nd.npar, cols = nd.cols;
    const int total_chunks = (int)((cols + kKC - 1) / kKC);
    const int cbeg = (int)(((int64_t)total_chunks * it.pad_) / it.begin);
    const int cend = (int)(((int64_t)total_chunks * (it.pad_ + 1)) / it.begin);
    const int nch = cend - cbeg;
    const void* tmx = tmaps + (int64_t)nd.tm_x * 128;
    const void* tmvh = tmaps + (int64_t)nd.tm_v * 128;
    const void* tmvl = tmaps + (int64_t)(nd.tm_v + 1) * 128;

    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < kXStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&x_full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_addr(&x_empty[s])));
        }
        for (int s = 0; s < kVStages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&v_full[s])));
        for (int t = 0; t < kTmStages; ++t) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_addr(&tm_full[t])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&freed[t])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&done_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    bool ok = true;

    if (warp == 0 || warp == 6) {
        // ---------------- producers (one thread each): X (warp 0) and V^T (warp 6). With a
        // test's injected fault they issue no loads, so the consumers' bounded waits run out.
        // Before leaving, each waits (bounded) for its last loads to land, so no copy is in
        // flight when the CTA exits, whatever happened to the consumers.
        if (lane == 0 && !inject) {
            const bool isx = warp == 0;
            const int S = isx ? kXStages : kVStages;
            uint64_t* full = isx ? x_full : v_full;
            uint64_t* empty = isx ? x_empty : freed;
            if (isx) {
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmx) : "memory");
            } else {
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmvh) : "memory");
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmvl) : "memory");
            }
            uint64_t policy;
            if (isx) asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
            else asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(policy));
            int issued = 0;
            for (int c = 0; c < nch && ok; ++c) {
                const int s = c % S;
                if (c >= S) ok = mbar_wait(smem_addr(&empty[s]), (uint32_t)((c / S - 1) & 1));
                if (!ok) break;
                const int k0 = (cbeg + c) * kKC;
                const uint32_t bar = smem_addr(&full[s]);
                if (isx) {
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kRawX)
                                 : "memory");
                    tma_load_2d_hint(smem_addr(xring + s * kRawX), tmx, k0, (int)row0, bar, policy);
                } else {
                    unsigned char* st = vring + s * 2 * kRawV;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(2 * kRawV)
                                 : "memory");
                    tma_load_2d_hint(smem_addr(st), tmvh, k0, rep0, bar, policy);
                    tma_load_2d_hint(smem_addr(st + kRawV), tmvl, k0, rep0, bar, policy);
                }
                issued = c + 1;
            }
            for (int c = issued > S ? issued - S : 0; c < issued; ++c)
                if (!mbar_wait(smem_addr(&full[c % S]), (uint32_t)((c / S) & 1))) ok = false;
        }
        __syncwarp();
    } else if (warp <= 4) {
        // ---------------- converters: thread = row q4 * 32 + lane of the tile (its TMEM lane)
        const int q4 = warp & 3;
        const int r = q4 * 32 + lane;
        const uint32_t lane_base = (uint32_t)(q4 * 32) << 16;
        for (int c = 0; c < nch && ok; ++c) {
            const int s = c % kXStages, t = c % kTmStages;
            ok = mbar_wait(smem_addr(&x_full[s]), (uint32_t)((c / kXStages) & 1));
            if (ok && c >= kTmStages) ok = mbar_wait(smem_addr(&freed[t]), (uint32_t)((c / kTmStages - 1) & 1));
            if (!ok) break;
            const unsigned char* rowp = xring + s * kRawX + (r >> 3) * 1024 + (r & 7) * 128;
            float4 v[8];
#pragma unroll
            for (int g = 0; g < 8; ++g) v[g] = *reinterpret_cast<const float4*>(rowp + ((g ^ (r & 7)) << 4));
            // this thread's reads of the stage are done (arrive releases them)
            mbar_arrive(smem_addr(&x_empty[s]));
            uint32_t hi[32], lo[32];
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                const float x[4] = {v[g].x, v[g].y, v[g].z, v[g].w};
#pragma unroll
                for (int q = 0; q < 4; ++q) tf32_split(x[q], hi[4 * g + q], lo[4 * g + q]);
            }
            const uint32_t col = (uint32_t)(kTN + 64 * t);
            tmem_store32(tmem + lane_base + col, hi);
            tmem_store32(tmem + lane_base + col + 32, lo);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            // one converter also waits for the chunk's V^T tiles, so that tm_full covers them
            if (warp == 1 && lane == 0) ok = mbar_wait(smem_addr(&v_full[t]), (uint32_t)((c / kTmStages) & 1));
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (ok && lane == 0) mbar_arrive(smem_addr(&tm_full[t]));
        }
    } else if (lane == 0) {
        // ---------------- MMA issue (warp 5, one thread)
        for (int c = 0; c < nch && ok; ++c) {
            const int t = c % kTmStages, sv = t;
            ok = mbar_wait(smem_addr(&tm_full[t]), (uint32_t)((c / kTmStages) & 1));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned char* st = vring + sv * 2 * kRawV;
            const uint32_t a_hi = tmem + (uint32_t)(kTN + 64 * t), a_lo = a_hi + 32;
            const uint32_t aop[3] = {a_hi, a_hi, a_lo};
            const unsigned char* bop[3] = {st, st + kRawV, st};
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int ks = 0; ks < kKC / 8; ++ks) {
                    const uint32_t at = aop[p] + ks * 8;
                    const uint64_t bd = smem_desc_sw128(smem_addr(bop[p]) + ks * 32);
                    const uint32_t acc = (c > 0 || p > 0 || ks > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, q;\n\t}" ::"r"(tmem),
                        "r"(at), "l"(bd), "r"(kIdesc), "r"(acc));
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&freed[t])));
            if (c == nch - 1)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(&done_bar)));
        }
    }
    if (!ok && (lane == 0)) atomicExch(err, DEVERR_TIMEOUT);

    if (warp >= 1 && warp <= 4 && ok && nch > 0) {
        // ---------------- epilogue: W^T[rep][row] from TMEM lanes 32 (warp % 4) .. + 31
        const bool done = mbar_wait(smem_addr(&done_bar), 0u);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!done) {
            if (lane == 0) atomicExch(err, DEVERR_TIMEOUT);
        } else {
            const int q4 = warp & 3;
            const int64_t row = row0 + q4 * 32 + lane;
#pragma unroll
            for (int cc = 0; cc < kTN / 16; ++cc) {
                uint32_t v[16];
                const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(cc * 16);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < npar) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int rep = rep0 + cc * 16 + j;
                        if (rep < R) {
                            float* dst = &ws[nd.w_off + (int64_t)rep * npar + row];
                            if (it.begin > 1)
                                atomicAdd(dst, __uint_as_float(v[j]));  // K split: partial sums
                            else
                                *dst = __uint_as_float(v[j]);
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 5) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ---------------------------------------------------------------------------
// Grouped-tensor variant (tnsk_rung, the grouping of Sec. 4.1): X(row, col) =
// sum_s A(.., s, ..) B(.., s, ..) is never stored. Rows are (i1, i2) (i2 fastest),
// columns (j1, j2) (j2 fastest, its dim a multiple of 32, so a 32-column chunk has
// one j1); A's entry (i1, s, j1) is at i1 ai + j1 aj + s as, B's (i2, s, j2) at
// i2 bi + j2 bj + s bs. The B factor is copied once per CTA into shared memory as
// [i2][s][j2] rows padded to 4 mod 32 floats (the distinct rows of one 16-byte load
// fall in distinct banks); the converters form their row's 32 entries of each chunk
// (FP32 fmaf over s in ascending order: the values contract_pairs writes), split
// them into TF32 hi / lo and store them to tensor memory as the streaming kernel
// does; only the V^T tiles arrive by TMA. Same warp roles, barriers and epilogue.
// ---------------------------------------------------------------------------
namespace {
// deeper rings than the streaming kernel's: 4 V^T stages (its X stages are not needed)
// and 3 operand stages (64 accumulator + 3 x 64 operand columns = the 256 allocated)
constexpr int kRungRaw = 4;
constexpr int kRungTm = 3;
constexpr int kRungRing = kRungRaw * 2 * kRawV;  // V^T hi + lo per stage
constexpr int kRungMmaWarp = 9;  // warps: 0 producer, 1-8 converters, 9 TMEM and MMA

// x[j] = sum_{s < SN} A(s) B(s, j) for 16 consecutive columns j (fma in ascending s, two
// columns per packed FP32 FMA; each half rounds like fmaf): the A terms at a + s (staged
// in shared memory, kSA) or a + s a_s (global), the B row at b + s nj2 (shared, 16-byte
// aligned).
template <int SN, bool kSA>
__device__ __forceinline__ void rung_entries(const float* a, int a_s, const float* b, int nj2, float2 (&x)[8]) {
    float av[SN];
#pragma unroll
    for (int s = 0; s < SN; ++s) av[s] = kSA ? a[s] : __ldg(a + (int64_t)s * a_s);
#pragma unroll
    for (int s = 0; s < SN; ++s) {
        const float4* bq = reinterpret_cast<const float4*>(b + s * nj2);
        const float2 aa = make_float2(av[s], av[s]);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const float4 v = bq[g];
            x[2 * g] = __ffma2_rn(aa, make_float2(v.x, v.y), x[2 * g]);
            x[2 * g + 1] = __ffma2_rn(aa, make_float2(v.z, v.w), x[2 * g + 1]);
        }
    }
}

}  // namespace

__global__ void __launch_bounds__(320, 2) m2_gemm_tc_rung_kernel(const M2Node* __restrict__ nodes,
                                                                 const M2Net* __restrict__ nets,
                                                                 const M2Item* __restrict__ items,
                                                                 float* __restrict__ ws,
                                                                 const unsigned char* __restrict__ tmaps,
                                                                 int* __restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t raw_full[kRungRaw], raw_empty[kRungRaw];
    __shared__ __align__(8) uint64_t tm_full[kRungTm], tm_empty[kRungTm];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_base;
    unsigned char* raw = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    float* sB = reinterpret_cast<float*>(raw + kRungRing);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const M2Item it = items[blockIdx.x];
    const M2Node& nd = nodes[it.node];
    const M2Net& N = nets[nd.net];
    const int R = N.R;
    const int64_t row0 = (int64_t)it.a * kTM;
    const int rep0 = it.b * kTN;
    const int64_t npar = nd.npar, cols = nd.cols;
    const int total_chunks = (int)((cols + kKC - 1) / kKC);
    const int cbeg = (int)(((int64_t)total_chunks * it.pad_) / it.begin);
    const int cend = (int)(((int64_t)total_chunks * (it.pad_ + 1)) / it.begin);
    const int nch = cend - cbeg;
    const void* tmvh = tmaps + (int64_t)nd.tm_v * 128;
    const void* tmvl = tmaps + (int64_t)(nd.tm_v + 1) * 128;
    const int ni2 = nd.rn_i2, nj2 = nd.rn_j2, sn = nd.rs;
    const int bp = sn * nj2 + 4;  // padded B row (floats)

    // the B factor, all threads: sB[i2 * bp + s * nj2 + j2] = B(i2, s, j2), several loads
    // in flight per thread
    {
        const float* __restrict__ Bg = nd.rB;
        const int per_i2 = sn * nj2;
        constexpr int kU = 4;
        if (nd.r_bj == 1 && nd.r_bs == nj2 && nd.r_bi == per_i2 && ((uintptr_t)Bg & 15) == 0) {
            // B(i2, s, j2) at i2 per_i2 + s nj2 + j2: contiguous rows, 16-byte copies
            const int per4 = per_i2 / 4, total4 = ni2 * per4;
            for (int q0 = tid; q0 < total4; q0 += kU * blockDim.x) {
                float4 v[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int q = q0 + u * blockDim.x;
                    v[u] = q < total4 ? __ldg(reinterpret_cast<const float4*>(Bg) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int q = q0 + u * blockDim.x;
                    if (q < total4) {
                        const int i2 = q / per4;
                        *reinterpret_cast<float4*>(sB + i2 * bp + 4 * (q - i2 * per4)) = v[u];
                    }
                }
            }
        } else {
            const int total = ni2 * per_i2;
            for (int q0 = tid; q0 < total; q0 += kU * blockDim.x) {
                float v[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int q = q0 + u * blockDim.x;
                    float x = 0.f;
                    if (q < total) {
                        const int i2 = q / per_i2, rem = q - i2 * per_i2;
                        const int sv = rem / nj2, j2 = rem - sv * nj2;
                        x = __ldg(Bg + (int64_t)i2 * nd.r_bi + (int64_t)sv * nd.r_bs + (int64_t)j2 * nd.r_bj);
                    }
                    v[u] = x;
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int q = q0 + u * blockDim.x;
                    if (q < total) {
                        const int i2 = q / per_i2;
                        sB[i2 * bp + (q - i2 * per_i2)] = v[u];
                    }
                }
            }
        }
    }
    // the A rows of the tile's i1 range, when the plan staged them: sA[(i1 - i1_lo) sn nj1 +
    // j1 sn + s] = A(i1, s, j1), so a chunk's terms are sn consecutive floats
    const int nj1 = nd.rn_j1;
    const int i1_lo = (int)(row0 / ni2);
    float* sA = sB + ni2 * bp;
    if (nd.r_astage) {
        const int64_t last = (row0 + kTM - 1 < npar ? row0 + kTM - 1 : npar - 1);
        const int cnt = (int)(last / ni2) - i1_lo + 1;
        const int per_i1 = sn * nj1, total = cnt * per_i1;
        for (int q = tid; q < total; q += blockDim.x) {
            const int di = q / per_i1, rem = q - di * per_i1;
            const int j1 = rem / sn, sv = rem - j1 * sn;
            sA[q] = __ldg(nd.rA + (int64_t)(i1_lo + di) * nd.r_ai + (int64_t)j1 * nd.r_aj + (int64_t)sv * nd.r_as);
        }
    }
    if (warp == kRungMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int st = 0; st < kRungRaw; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&raw_full[st])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&raw_empty[st])));
        }
        for (int t = 0; t < kRungTm; ++t) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_addr(&tm_full[t])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&tm_empty[t])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&done_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    bool ok = true;

    if (warp == 0) {
        // ---------------- producer (one thread): the V^T hi / lo tiles of each chunk
        if (lane == 0) {
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmvh) : "memory");
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmvl) : "memory");
            for (int c = 0; c < nch && ok; ++c) {
                const int st = c % kRungRaw;
                if (c >= kRungRaw)
                    ok = mbar_wait(smem_addr(&raw_empty[st]), (uint32_t)((c / kRungRaw - 1) & 1));
                if (!ok) break;
                const int k0 = (cbeg + c) * kKC;
                unsigned char* stp = raw + st * 2 * kRawV;
                const uint32_t bar = smem_addr(&raw_full[st]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(2 * kRawV)
                             : "memory");
                tma_load_2d(smem_addr(stp), tmvh, k0, rep0, bar);
                tma_load_2d(smem_addr(stp + kRawV), tmvl, k0, rep0, bar);
            }
        }
        __syncwarp();
    } else if (warp <= 8) {
        // ---------------- converters, two warps per TMEM lane quarter q4 = warp % 4 (the
        // quarter a warp may access), each forming 16 of a chunk's 32 columns (half hf).
        // TMEM lane q4 * 32 + lane holds tile row pr, a permutation that gives each group
        // of 4 lanes one i2 when n_i2 = 32 (4 i1 x 32 i2 per tile), so a warp's B reads hit
        // 8 addresses, each a 4-lane broadcast
        const int q4 = warp & 3, hf = (warp - 1) >> 2;
        const int pr = (lane & 3) * 32 + q4 * 8 + (lane >> 2);
        const int64_t row = row0 + pr;
        const bool live = row < npar;
        const int i1 = live ? (int)(row / ni2) : 0, i2 = live ? (int)(row - (int64_t)i1 * ni2) : 0;
        const float* __restrict__ Arow = nd.rA + (int64_t)i1 * nd.r_ai;
        const float* Brow = sB + i2 * bp + 16 * hf;
        const uint32_t lane_base = (uint32_t)(q4 * 32) << 16;
        for (int c = 0; c < nch && ok; ++c) {
            const int t = c % kRungTm;
            if (c >= kRungTm) ok = mbar_wait(smem_addr(&tm_empty[t]), (uint32_t)((c / kRungTm - 1) & 1));
            if (!ok) break;
            const int k0 = (cbeg + c) * kKC;
            const int j1 = k0 / nj2, j20 = k0 - j1 * nj2;
            float2 x2[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) x2[j] = make_float2(0.f, 0.f);
            if (live) {
                const bool sa = nd.r_astage != 0;
                const float* Aj = sa ? sA + (i1 - i1_lo) * sn * nj1 + j1 * sn : Arow + (int64_t)j1 * nd.r_aj;
                const float* Bj = Brow + j20;
                switch (sn) {  // the shared dim as a compile-time trip count: loads hoisted
#define TNSK_RUNG_SN(n)                                                   \
    case n:                                                               \
        if (sa)                                                           \
            rung_entries<n, true>(Aj, 1, Bj, nj2, x2);                    \
        else                                                              \
            rung_entries<n, false>(Aj, nd.r_as, Bj, nj2, x2);             \
        break;
                    TNSK_RUNG_SN(1) TNSK_RUNG_SN(2) TNSK_RUNG_SN(3) TNSK_RUNG_SN(4) TNSK_RUNG_SN(5) TNSK_RUNG_SN(6)
                    TNSK_RUNG_SN(7) TNSK_RUNG_SN(8) TNSK_RUNG_SN(9) TNSK_RUNG_SN(10) TNSK_RUNG_SN(11)
                    TNSK_RUNG_SN(12) TNSK_RUNG_SN(13) TNSK_RUNG_SN(14) TNSK_RUNG_SN(15) TNSK_RUNG_SN(16)
#undef TNSK_RUNG_SN
                    default: break;
                }
            }
            float x[16];
#pragma unroll
            for (int j = 0; j < 8; ++j) x[2 * j] = x2[j].x, x[2 * j + 1] = x2[j].y;
            uint32_t hi[16], lo[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) tf32_split(x[j], hi[j], lo[j]);
            // the previous chunk's stores had this chunk's arithmetic to complete: wait for
            // them and hand that stage to the MMA only now, then store this chunk
            if (c > 0) {
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_addr(&tm_full[(c - 1) % kRungTm]));
            }
            const uint32_t col = (uint32_t)(kTN + 64 * t + 16 * hf);
            tmem_store16(tmem + lane_base + col, hi);
            tmem_store16(tmem + lane_base + col + 32, lo);
        }
        if (ok && nch > 0) {
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&tm_full[(nch - 1) % kRungTm]));
        }
    } else if (lane == 0) {
        // ---------------- MMA issue (warp 9, one thread)
        for (int c = 0; c < nch && ok; ++c) {
            const int st = c % kRungRaw, t = c % kRungTm;
            ok = mbar_wait(smem_addr(&tm_full[t]), (uint32_t)((c / kRungTm) & 1));
            if (ok) ok = mbar_wait(smem_addr(&raw_full[st]), (uint32_t)((c / kRungRaw) & 1));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned char* stp = raw + st * 2 * kRawV;
            const uint32_t a_hi = tmem + (uint32_t)(kTN + 64 * t), a_lo = a_hi + 32;
            const uint32_t aop[3] = {a_hi, a_hi, a_lo};
            const unsigned char* bop[3] = {stp, stp + kRawV, stp};
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int ks = 0; ks < kKC / 8; ++ks) {
                    const uint32_t at = aop[p] + ks * 8;
                    const uint64_t bd = smem_desc_sw128(smem_addr(bop[p]) + ks * 32);
                    const uint32_t acc = (c > 0 || p > 0 || ks > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, q;\n\t}" ::"r"(tmem),
                        "r"(at), "l"(bd), "r"(kIdesc), "r"(acc));
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&tm_empty[t])));
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&raw_empty[st])));
            if (c == nch - 1)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(&done_bar)));
        }
    }
    if (!ok && (lane == 0)) atomicExch(err, DEVERR_TIMEOUT);

    if (warp >= 1 && warp <= 8 && ok && nch > 0) {
        // ---------------- epilogue: W^T[rep][row] from TMEM lanes 32 (warp % 4) .. + 31,
        // reps [32 hf, 32 hf + 32) per warp
        const bool done = mbar_wait(smem_addr(&done_bar), 0u);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!done) {
            if (lane == 0) atomicExch(err, DEVERR_TIMEOUT);
        } else {
            const int q4 = warp & 3, hf = (warp - 1) >> 2;
            const int64_t row = row0 + (lane & 3) * 32 + q4 * 8 + (lane >> 2);  // the converters' row map
#pragma unroll
            for (int cc = 2 * hf; cc < 2 * hf + 2; ++cc) {
                uint32_t v[16];
                const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(cc * 16);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < npar) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int rep = rep0 + cc * 16 + j;
                        if (rep < R) {
                            float* dst = &ws[nd.w_off + (int64_t)rep * npar + row];
                            if (it.begin > 1)
                                atomicAdd(dst, __uint_as_float(v[j]));  // K split: partial sums
                            else
                                *dst = __uint_as_float(v[j]);
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kRungMmaWarp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

size_t m2_gemm_rung_smem(size_t b_bytes) { return 1024 + (size_t)kRungRing + b_bytes; }

cudaError_t launch_m2_gemm_tc_rung(int n, const M2Node* nodes, const M2Net* nets, const M2Item* items, float* ws,
                                   const unsigned char* tmaps, int* err, size_t smem, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    cudaFuncSetAttribute(m2_gemm_tc_rung_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    m2_gemm_tc_rung_kernel<<<n, 320, smem, s>>>(nodes, nets, items, ws, tmaps, err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// BF16 variant (TNSK_PREC_BF16, tensors stored as BF16): the same product with
// BF16 operands and FP32 accumulation in tensor memory (tcgen05.mma kind::f16).
// X (row-major BF16, parent mode first, cols a multiple of 8) arrives by TMA as it
// is stored: per K-chunk of 64 columns a 128 x 64 tile (128-byte rows, 128-byte
// swizzle). V^T is stored by the V build as three BF16 parts V = Vh + Vm + Vl
// (each the BF16 rounding of what the previous parts leave; together within
// 2^-24 of V), so W = X Vh + X Vm + X Vl is the product with V at FP32 precision and
// X exactly as stored: three MMA passes per chunk, both operands read from shared
// memory, no conversion of X at all. Half the bytes of X of the FP32 path.
//   warp 0     producer: four TMA loads per chunk (X, Vh, Vm, Vl) into a ring
//   warp 1     tensor memory allocation and MMA issue
//   warps 2-5  epilogue (each the TMEM lane quarter warp % 4)
// ---------------------------------------------------------------------------
namespace {
constexpr int kBfKC = 64;                                // columns per chunk (4 MMAs of K = 16)
constexpr int kBfStages = 2;                             // two CTAs per SM
constexpr int kBfX = kTM * 128;                          // 128 rows x 128 B
constexpr int kBfV = kTN * 128;                          // 64 rows x 128 B, one part
constexpr int kBfStage = kBfX + 3 * kBfV;                // 40 KiB
constexpr int kBfSmem = kBfStages * kBfStage + 1024;
// Instruction descriptor: D = F32, A = B = BF16, both K-major, N = 64, M = 128.
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                                ((uint32_t)(kTM >> 4) << 24);
}  // namespace

__global__ void __launch_bounds__(192, 2) m2_gemm_bf16_kernel(const M2Node* __restrict__ nodes,
                                                              const M2Net* __restrict__ nets,
                                                              const M2Item* __restrict__ items,
                                                              float* __restrict__ ws,
                                                              const unsigned char* __restrict__ tmaps,
                                                              int* __restrict__ err, int inject) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kBfStages], empty[kBfStages];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_base;
    unsigned char* ring = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const M2Item it = items[blockIdx.x];
    const M2Node& nd = nodes[it.node];
    const M2Net& N = nets[nd.net];
    const int R = N.R;
    const int64_t row0 = (int64_t)it.a * kTM;
    const int rep0 = it.b * kTN;
    const int64_t npar = nd.npar, cols = nd.cols;
    const int total_chunks = (int)((cols + kBfKC - 1) / kBfKC);
    const int cbeg = (int)(((int64_t)total_chunks * it.pad_) / it.begin);
    const int cend = (int)(((int64_t)total_chunks * (it.pad_ + 1)) / it.begin);
    const int nch = cend - cbeg;
    const void* tmx = tmaps + (int64_t)nd.tm_x * 128;
    const void* tmv[3] = {tmaps + (int64_t)nd.tm_v * 128, tmaps + (int64_t)(nd.tm_v + 1) * 128,
                          tmaps + (int64_t)(nd.tm_v + 2) * 128};

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(kTN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < kBfStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&done_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0 && !inject) {  // a test's injected fault: no loads (the waits below run out)
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmx) : "memory");
            for (int p = 0; p < 3; ++p)
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmv[p]) : "memory");
            for (int c = 0; c < nch && ok; ++c) {
                const int s = c % kBfStages;
                if (c >= kBfStages) ok = mbar_wait(smem_addr(&empty[s]), (uint32_t)((c / kBfStages - 1) & 1));
                if (!ok) break;
                const int k0 = (cbeg + c) * kBfKC;
                unsigned char* st = ring + s * kBfStage;
                const uint32_t bar = smem_addr(&full[s]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBfStage)
                             : "memory");
                tma_load_2d(smem_addr(st), tmx, k0, (int)row0, bar);
                for (int p = 0; p < 3; ++p) tma_load_2d(smem_addr(st + kBfX + p * kBfV), tmv[p], k0, rep0, bar);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            for (int c = 0; c < nch && ok; ++c) {
                const int s = c % kBfStages;
                ok = mbar_wait(smem_addr(&full[s]), (uint32_t)((c / kBfStages) & 1));
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned char* st = ring + s * kBfStage;
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int ks = 0; ks < kBfKC / 16; ++ks) {
                        const uint64_t ad = smem_desc_sw128(smem_addr(st) + ks * 32);
                        const uint64_t bd = smem_desc_sw128(smem_addr(st + kBfX + p * kBfV) + ks * 32);
                        const uint32_t acc = (c > 0 || p > 0 || ks > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}" ::"r"(tmem),
                            "l"(ad), "l"(bd), "r"(kIdescBf16), "r"(acc));
                    }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(&empty[s])));
                if (c == nch - 1)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_addr(&done_bar)));
            }
        }
        __syncwarp();
    }
    if (!ok && lane == 0) atomicExch(err, DEVERR_TIMEOUT);

    if (warp >= 2 && nch > 0) {
        // epilogue: W^T[rep][row] from TMEM lanes 32 (warp % 4) .. + 31
        const bool done = mbar_wait(smem_addr(&done_bar), 0u);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!done) {
            if (lane == 0) atomicExch(err, DEVERR_TIMEOUT);
        } else {
            const int q4 = warp & 3;
            const int64_t row = row0 + q4 * 32 + lane;
#pragma unroll
            for (int cc = 0; cc < kTN / 16; ++cc) {
                uint32_t v[16];
                const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(cc * 16);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < npar) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int rep = rep0 + cc * 16 + j;
                        if (rep < R) {
                            float* dst = &ws[nd.w_off + (int64_t)rep * npar + row];
                            if (it.begin > 1)
                                atomicAdd(dst, __uint_as_float(v[j]));  // K split: partial sums
                            else
                                *dst = __uint_as_float(v[j]);
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTN));
}

cudaError_t launch_m2_gemm_bf16(int n, const M2Node* nodes, const M2Net* nets, const M2Item* items, float* ws,
                                const unsigned char* tmaps, int* err, int inject, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    cudaFuncSetAttribute(m2_gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBfSmem);
    m2_gemm_bf16_kernel<<<n, 192, kBfSmem, s>>>(nodes, nets, items, ws, tmaps, err, inject);
    return cudaGetLastError();
}

cudaError_t launch_m2_gemm_tc(int n, const M2Node* nodes, const M2Net* nets, const M2Item* items,
                              const uint32_t* tabs, float* ws, const unsigned char* tmaps, int* err, bool stream,
                              int inject, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (stream) {
        cudaFuncSetAttribute(m2_gemm_tc_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kStreamSmem);
        m2_gemm_tc_stream_kernel<<<n, kStreamThreads, kStreamSmem, s>>>(nodes, nets, items, ws, tmaps, err, inject);
    } else {
        cudaFuncSetAttribute(m2_gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        m2_gemm_tc_kernel<<<n, 128, kSmemBytes, s>>>(nodes, nets, items, tabs, ws, err);
    }
    return cudaGetLastError();
}

}  // namespace tnsk
