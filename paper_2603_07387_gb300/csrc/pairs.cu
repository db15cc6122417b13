// pairs.cu -- exact contraction of pairs of tensors into one tensor each (the
// normalisations of Sec. 4.1: grouping two tensors with their shared contractions
// summed exactly; several contractions between the pair and a third tensor become
// one mode of the grouped tensor by a reshape of adjacent output modes). Used to
// turn two tensor trains joined on their physical legs (a cyclic ladder) into an
// acyclic chain for method 2: M_k[a, b, c, d] = sum_s A_k[a, s, c] B_k[b, s, d].
//
// out[i] = sum over the shared multi-index s of A[.., s, ..] * B[.., s, ..], FP32
// products summed in FP32. Rows are every output mode but the last; a warp works on
// 32 rows at a time, lanes along the last output mode (coalesced stores). FP32
// inputs with 32-bit offsets take a path that decodes the 32 rows at once (one per
// lane, then shuffles), reads the (A, B) offsets of the shared combinations from a
// small shared-memory table, and, when the 32 rows share their B operands (the
// tensor-train merge: consecutive rows differ in an A mode only), keeps each lane's
// B terms in registers across the rows (16-byte stores when the last mode runs
// along B only). Other inputs take a general path. The output is written once.
#include <algorithm>
#include <string>
#include <vector>

#include "ctx.cuh"
#include "kernels.cuh"

namespace tnsk {
namespace {

constexpr int kMaxOut = 2 * TNSK_MAX_ORDER;
constexpr int kMaxShared = TNSK_MAX_ORDER;
constexpr int kShTable = 256;   // shared combinations tabulated in shared memory (2 KiB)
constexpr int kRegTerms = 16;   // shared combinations held in registers when rows reuse B

struct PairDesc {
    const void* A;
    const void* B;
    float* out;
    int64_t out_numel, sh_numel;
    int64_t out_dim[kMaxOut], a_out_str[kMaxOut], b_out_str[kMaxOut];
    int64_t sh_dim[kMaxShared], a_sh_str[kMaxShared], b_sh_str[kMaxShared];
    int32_t n_out, n_sh, a_dtype, b_dtype;
    int32_t fast;  // FP32 inputs, every offset below 2^31: the 32-bit path
    int32_t pad_;
};
static_assert(sizeof(PairDesc) % 8 == 0, "descriptor copied as 8-byte words");

// Rows base + i (i < nr) whose B operands agree, NS shared terms: each lane holds its
// output column's B terms and the A offsets in registers, four rows at a time.
template <int NS>
__device__ __forceinline__ void rows_same_b(const float* __restrict__ A, const float* __restrict__ B,
                                            float* __restrict__ out, const int2* __restrict__ tab, int ra, int rb,
                                            int la, int lb, int L, int nr, int base, int lane) {
    int ta[NS];
    float bv[NS];
    const bool live = lane < L;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        const int2 t = tab[q];
        ta[q] = t.x + lane * la;
        bv[q] = live ? __ldg(B + rb + lane * lb + t.y) : 0.f;
    }
    for (int i = 0; i < nr; i += 4) {
        int pa[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) pa[k] = __shfl_sync(0xffffffffu, ra, min(i + k, nr - 1));
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (live) {
#pragma unroll
            for (int q = 0; q < NS; ++q)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[k] += __ldg(A + pa[k] + ta[q]) * bv[q];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (i + k < nr) out[(int64_t)(base + i + k) * L + lane] = acc[k];
        }
    }
}

// The same rows when the last output mode runs along B only (la = 0, lb = 1) with
// 4 <= L <= 32, L % 4 == 0: 8 lanes per row, 4 consecutive columns per lane (16-byte
// stores), 4 rows per pass of the warp. The A terms do not depend on the column: lane
// i loads row base + i's NS terms once, and each row takes them by shuffle, so no
// load waits inside the row loop.
template <int NS>
__device__ __forceinline__ void rows_same_b_v4(const float* __restrict__ A, const float* __restrict__ B,
                                               float* __restrict__ out, const int2* __restrict__ tab, int ra,
                                               int rb, int L, int nr, int base, int lane) {
    const int r4 = lane >> 3, c = (lane & 7) * 4;
    const bool live = c < L;
    float av[NS];
    float bv[NS][4];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        const int2 t = tab[q];
        av[q] = lane < nr ? __ldg(A + ra + t.x) : 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[q][j] = live ? __ldg(B + rb + c + j + t.y) : 0.f;
    }
    for (int i = 0; i < nr; i += 4) {
        const int row = i + r4;
        // two columns per packed FP32 FMA (each half rounds like fmaf)
        float2 acc01 = make_float2(0.f, 0.f), acc23 = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const float a = __shfl_sync(0xffffffffu, av[q], row & 31);
            const float2 aa = make_float2(a, a);
            acc01 = __ffma2_rn(aa, make_float2(bv[q][0], bv[q][1]), acc01);
            acc23 = __ffma2_rn(aa, make_float2(bv[q][2], bv[q][3]), acc23);
        }
        if (live && row < nr)
            *reinterpret_cast<float4*>(out + (int64_t)(base + row) * L + c) =
                make_float4(acc01.x, acc01.y, acc23.x, acc23.y);
    }
}

}  // namespace

// kFast: the jobs that take the 32-bit FP32 path (fast flag, at most kShTable shared
// combinations); otherwise the rest. The two are separate kernels so the general
// path's 64-bit state does not raise the fast path's register count.
template <bool kFast>
__global__ void __launch_bounds__(256, 4) contract_pairs_kernel(const PairDesc* __restrict__ jobs) {
    __shared__ PairDesc d;
    __shared__ int2 tab[kShTable];  // (A, B) offsets of the shared combinations, 32-bit path
    {  // the job's descriptor, copied by the whole block
        const uint64_t* src = reinterpret_cast<const uint64_t*>(jobs + blockIdx.y);
        uint64_t* dst = reinterpret_cast<uint64_t*>(&d);
        for (int i = threadIdx.x; i < (int)(sizeof(PairDesc) / 8); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int64_t nsh = d.sh_numel;
    const bool fast = d.fast && nsh <= kShTable;
    if (fast != kFast) return;
    auto shared_offsets = [&](int64_t s, int64_t& sa, int64_t& sb) {
        sa = sb = 0;
        for (int j = d.n_sh - 1; j >= 0; --j) {
            const int64_t q = s / d.sh_dim[j];
            const int64_t dj = s - q * d.sh_dim[j];
            s = q;
            sa += dj * d.a_sh_str[j];
            sb += dj * d.b_sh_str[j];
        }
    };
    if (kFast)
        for (int64_t q = threadIdx.x; q < nsh; q += blockDim.x) {
            int64_t sa, sb;
            shared_offsets(q, sa, sb);
            tab[q] = make_int2((int)sa, (int)sb);
        }
    __syncthreads();
    if (d.out_numel == 0) return;
    const int lane = threadIdx.x & 31;
    if constexpr (kFast) {
        const float* __restrict__ A = static_cast<const float*>(d.A);
        const float* __restrict__ B = static_cast<const float*>(d.B);
        const int last = d.n_out - 1;
        const int L = last >= 0 ? (int)d.out_dim[last] : 1;
        const int la = last >= 0 ? (int)d.a_out_str[last] : 0, lb = last >= 0 ? (int)d.b_out_str[last] : 0;
        const int rows = (int)(d.out_numel / L);
        const int ns = (int)nsh;
        const int nw = gridDim.x * (blockDim.x >> 5);
        const bool v4 = la == 0 && lb == 1 && L >= 4 && L <= 32 && L % 4 == 0 && ((uintptr_t)d.out & 15) == 0;
        for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < rows; base += nw * 32) {
            int ra = 0, rb = 0;  // offsets of row base + lane
            {
                unsigned rem = (unsigned)(base + lane);
                for (int j = last - 1; j >= 0; --j) {
                    const unsigned dim = (unsigned)d.out_dim[j];
                    const unsigned q = rem / dim;
                    const int dj = (int)(rem - q * dim);
                    rem = q;
                    ra += dj * (int)d.a_out_str[j];
                    rb += dj * (int)d.b_out_str[j];
                }
            }
            const int nr = min(32, rows - base);
            const bool same_b = __all_sync(0xffffffffu, rb == __shfl_sync(0xffffffffu, rb, 0));
            if (same_b && v4 && ns <= 8) {
                switch (ns) {
#define TNSK_ROWS(n) \
    case n: rows_same_b_v4<n>(A, B, d.out, tab, ra, rb, L, nr, base, lane); break;
                    TNSK_ROWS(1) TNSK_ROWS(2) TNSK_ROWS(3) TNSK_ROWS(4) TNSK_ROWS(5) TNSK_ROWS(6) TNSK_ROWS(7)
                    TNSK_ROWS(8)
#undef TNSK_ROWS
                    default: break;
                }
                continue;
            }
            if (same_b && L <= 32 && ns <= kRegTerms) {
                switch (ns) {
#define TNSK_ROWS(n) \
    case n: rows_same_b<n>(A, B, d.out, tab, ra, rb, la, lb, L, nr, base, lane); break;
                    TNSK_ROWS(1) TNSK_ROWS(2) TNSK_ROWS(3) TNSK_ROWS(4) TNSK_ROWS(5) TNSK_ROWS(6) TNSK_ROWS(7)
                    TNSK_ROWS(8) TNSK_ROWS(9) TNSK_ROWS(10) TNSK_ROWS(11) TNSK_ROWS(12) TNSK_ROWS(13)
                    TNSK_ROWS(14) TNSK_ROWS(15) TNSK_ROWS(16)
#undef TNSK_ROWS
                    default: break;
                }
                continue;
            }
            for (int i = 0; i < nr; ++i) {
                const int pa = __shfl_sync(0xffffffffu, ra, i), pb = __shfl_sync(0xffffffffu, rb, i);
                float* orow = d.out + (int64_t)(base + i) * L;
                for (int x = lane; x < L; x += 32) {
                    const int oa = pa + x * la, ob = pb + x * lb;
                    float acc = 0.f;
#pragma unroll 4
                    for (int q = 0; q < ns; ++q) {
                        const int2 t = tab[q];
                        acc += __ldg(A + oa + t.x) * __ldg(B + ob + t.y);
                    }
                    orow[x] = acc;
                }
            }
        }
    } else {
    // general path: any dtype, 64-bit offsets, the shared combinations decoded per term
    const int last = d.n_out - 1;
    const int64_t L = last >= 0 ? d.out_dim[last] : 1;
    const int64_t la = last >= 0 ? d.a_out_str[last] : 0, lb = last >= 0 ? d.b_out_str[last] : 0;
    const int64_t rows = d.out_numel / L;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += nwarps) {
        int64_t rem = row, ra = 0, rb = 0;
        for (int j = last - 1; j >= 0; --j) {
            const int64_t q = rem / d.out_dim[j];
            const int64_t dj = rem - q * d.out_dim[j];
            rem = q;
            ra += dj * d.a_out_str[j];
            rb += dj * d.b_out_str[j];
        }
        for (int64_t x = lane; x < L; x += 32) {
            const int64_t oa = ra + x * la, ob = rb + x * lb;
            float acc = 0.f;
            for (int64_t s = 0; s < nsh; ++s) {
                int64_t sa, sb;
                shared_offsets(s, sa, sb);
                acc += load_as<float>(d.A, d.a_dtype, oa + sa) * load_as<float>(d.B, d.b_dtype, ob + sb);
            }
            d.out[row * L + x] = acc;
        }
    }
    }
}

}  // namespace tnsk

using namespace tnsk;

struct tnsk_pairs {
    int device = 0;
    int sms = 1;
    int n = 0;
    bool any_fast = false, any_general = false;
    PairDesc* dev = nullptr;
    std::vector<int64_t> sizes;
};

namespace {

tnsk_status describe(tnsk_ctx* ctx, const tnsk_pair_job& jb, PairDesc& d) {
    if (!jb.A || !jb.B || !jb.out || (jb.n_shared > 0 && (!jb.a_modes || !jb.b_modes)))
        return ctx_fail(ctx, TNSK_ERR_INVALID, "contract_pairs: NULL argument");
    const tnsk_tensor& A = *jb.A;
    const tnsk_tensor& B = *jb.B;
    auto dtype_ok = [](int t) { return t == TNSK_F32 || t == TNSK_F64 || t == TNSK_BF16; };
    if (A.order < 0 || B.order < 0 || A.order > TNSK_MAX_ORDER || B.order > TNSK_MAX_ORDER || !dtype_ok(A.dtype) ||
        !dtype_ok(B.dtype) || (A.order > 0 && !A.dims) || (B.order > 0 && !B.dims) || !A.data || !B.data)
        return ctx_fail(ctx, TNSK_ERR_INVALID, "contract_pairs: bad tensor");
    if (jb.n_shared < 0 || jb.n_shared > A.order || jb.n_shared > B.order)
        return ctx_fail(ctx, TNSK_ERR_INVALID, "contract_pairs: n_shared");
    int64_t na = 1, nb = 1;
    for (int i = 0; i < A.order; ++i) {
        if (A.dims[i] < 0) return ctx_fail(ctx, TNSK_ERR_INVALID, "contract_pairs: negative dim");
        na *= A.dims[i];
    }
    for (int i = 0; i < B.order; ++i) {
        if (B.dims[i] < 0) return ctx_fail(ctx, TNSK_ERR_INVALID, "contract_pairs: negative dim");
        nb *= B.dims[i];
    }
    std::vector<int64_t> sa(A.order), sb(B.order);  // row-major strides
    int64_t s = 1;
    for (int i = A.order - 1; i >= 0; --i) sa[i] = s, s *= A.dims[i];
    s = 1;
    for (int i = B.order - 1; i >= 0; --i) sb[i] = s, s *= B.dims[i];
    std::vector<int> a_used(A.order, 0), b_used(B.order, 0);
    d = PairDesc{};
    d.A = A.data;
    d.B = B.data;
    d.out = jb.out;
    d.a_dtype = A.dtype;
    d.b_dtype = B.dtype;
    d.n_sh = jb.n_shared;
    d.sh_numel = 1;
    for (int j = 0; j < jb.n_shared; ++j) {
        const int a = jb.a_modes[j], b = jb.b_modes[j];
        if (a < 0 || a >= A.order || b < 0 || b >= B.order || a_used[a] || b_used[b] || A.dims[a] != B.dims[b])
            return ctx_fail(ctx, TNSK_ERR_INVALID, "contract_pairs: shared modes must be distinct and of equal dims");
        a_used[a] = b_used[b] = 1;
        d.sh_dim[j] = A.dims[a];
        d.a_sh_str[j] = sa[a];
        d.b_sh_str[j] = sb[b];
        if (A.dims[a] > 0 && d.sh_numel > ((int64_t)1 << 20) / A.dims[a])
            return ctx_fail(ctx, TNSK_ERR_UNSUPPORTED, "contract_pairs: above 2^20 shared index combinations");
        d.sh_numel *= A.dims[a];
    }
    // free modes: A's in order, then B's
    std::vector<int64_t> fdim, fa, fb;
    for (int i = 0; i < A.order; ++i)
        if (!a_used[i]) fdim.push_back(A.dims[i]), fa.push_back(sa[i]), fb.push_back(0);
    for (int i = 0; i < B.order; ++i)
        if (!b_used[i]) fdim.push_back(B.dims[i]), fa.push_back(0), fb.push_back(sb[i]);
    d.n_out = (int)fdim.size();
    d.fast = A.dtype == TNSK_F32 && B.dtype == TNSK_F32 && na < ((int64_t)1 << 31) && nb < ((int64_t)1 << 31);
    std::vector<int> seen(d.n_out, 0);
    d.out_numel = 1;
    for (int i = 0; i < d.n_out; ++i) {
        const int f = jb.out_perm ? jb.out_perm[i] : i;
        if (f < 0 || f >= d.n_out || seen[f]) return ctx_fail(ctx, TNSK_ERR_INVALID, "contract_pairs: out_perm");
        seen[f] = 1;
        d.out_dim[i] = fdim[f];
        d.a_out_str[i] = fa[f];
        d.b_out_str[i] = fb[f];
        if (fdim[f] > 0 && d.out_numel > ((int64_t)1 << 31) / fdim[f])
            return ctx_fail(ctx, TNSK_ERR_UNSUPPORTED, "contract_pairs: above 2^31 output entries");
        d.out_numel *= fdim[f];
    }
    return TNSK_OK;
}

}  // namespace

extern "C" {

tnsk_status tnsk_pairs_create(tnsk_ctx* ctx, int32_t n, const tnsk_pair_job* jobs, tnsk_pairs** out) {
    if (!out) return TNSK_ERR_INVALID;
    *out = nullptr;
    tnsk_status st = ctx_check(ctx);
    if (st != TNSK_OK) return st;
    if (n < 0 || n > 65535 || (n > 0 && !jobs)) return ctx_fail(ctx, TNSK_ERR_INVALID, "pairs: n in [0, 65535]");
    std::vector<PairDesc> h((size_t)n);
    for (int i = 0; i < n; ++i) {
        st = describe(ctx, jobs[i], h[(size_t)i]);
        if (st != TNSK_OK) return st;
    }
    tnsk_pairs* p = new tnsk_pairs();
    p->device = ctx->device;
    cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, ctx->device);
    p->sms = std::max(p->sms, 1);
    p->n = n;
    for (const PairDesc& d : h) {
        p->sizes.push_back(d.out_numel);
        const bool fast = d.fast && d.sh_numel <= kShTable;
        p->any_fast |= fast;
        p->any_general |= !fast;
    }
    if (n > 0) {
        if (cudaMalloc((void**)&p->dev, h.size() * sizeof(PairDesc)) != cudaSuccess ||
            cudaMemcpy(p->dev, h.data(), h.size() * sizeof(PairDesc), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(p->dev);
            delete p;
            return ctx_fail(ctx, TNSK_ERR_OOM, "pairs: descriptor upload");
        }
    }
    *out = p;
    return TNSK_OK;
}

tnsk_status tnsk_pairs_run(tnsk_ctx* ctx, tnsk_pairs* p) {
    tnsk_status st = ctx_check(ctx);
    if (st != TNSK_OK) return st;
    if (!p) return ctx_fail(ctx, TNSK_ERR_INVALID, "pairs: NULL");
    if (p->device != ctx->device) return ctx_fail(ctx, TNSK_ERR_INVALID, "pairs made on another device");
    if (p->n == 0) return TNSK_OK;
    int64_t most = 1;
    for (int64_t s : p->sizes) most = std::max(most, s);
    // blocks of 8 warps, warps striding over groups of 32 rows: about eight waves of
    // blocks (four per SM) over all jobs, so the per-block setup (descriptor, offset
    // table) is paid a few times per SM, not once per 8192 outputs
    const int64_t per_job = (8 * 4 * (int64_t)p->sms + p->n - 1) / p->n;
    const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>({(most + 8191) / 8192, per_job, 1024}));
    ctx->prof.begin(TNSK_K_PAIRS, ctx->stream);
    if (p->any_fast) contract_pairs_kernel<true><<<dim3(gx, (unsigned)p->n), 256, 0, ctx->stream>>>(p->dev);
    if (p->any_general) contract_pairs_kernel<false><<<dim3(gx, (unsigned)p->n), 256, 0, ctx->stream>>>(p->dev);
    ctx->prof.end(ctx->stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "contract_pairs_kernel");
    return TNSK_OK;
}

tnsk_status tnsk_pairs_destroy(tnsk_pairs* p) {
    if (!p) return TNSK_ERR_INVALID;
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    cudaFree(p->dev);
    delete p;
    return TNSK_OK;
}

tnsk_status tnsk_contract_pairs(tnsk_ctx* ctx, int32_t n, const tnsk_pair_job* jobs) {
    tnsk_pairs* p = nullptr;
    tnsk_status st = tnsk_pairs_create(ctx, n, jobs, &p);
    if (st != TNSK_OK) return st;
    st = tnsk_pairs_run(ctx, p);
    cudaStreamSynchronize(ctx->stream);
    tnsk_pairs_destroy(p);
    return st;
}

}  // extern "C"
