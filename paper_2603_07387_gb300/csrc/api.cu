// api.cu -- host side of the libtnsk C ABI: validation of the network and the
// parameters (Def. "Tensor contraction": u != v, n_u = n_v), planning of the
// launches, scratch management and error reporting. Every arithmetic step of
// the estimators runs in the kernels; the host only lays out descriptors.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.cuh"
#include "kernels.cuh"
#include "method2.cuh"
#include "normalize.cuh"
#include "plan.cuh"

using namespace tnsk;

namespace {

tnsk_status fail(tnsk_ctx* ctx, tnsk_status st, const std::string& msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

tnsk_status cuda_fail(tnsk_ctx* ctx, cudaError_t e, const char* where) {
    return fail(ctx, TNSK_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define TNSK_CUDA(call)                                       \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// Grows a ctx-owned device buffer to at least `bytes` (earlier work on the stream
// may still read the old one, so it is freed after a stream synchronisation).
tnsk_status ensure_buffer(tnsk_ctx* ctx, unsigned char*& buf, size_t& have, size_t bytes, const char* what) {
    if (bytes <= have) return TNSK_OK;
    size_t want = std::max(bytes, have + have / 2);
    want = (want + ((size_t)1 << 20) - 1) & ~(((size_t)1 << 20) - 1);
    if (buf) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
        cudaFree(buf);
        buf = nullptr;
        have = 0;
    }
    cudaError_t e = cudaMalloc((void**)&buf, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, TNSK_ERR_OOM, std::string(what) + " allocation of " + std::to_string(want) + " bytes failed");
    }
    have = want;
    return TNSK_OK;
}

tnsk_status ensure_scratch(tnsk_ctx* ctx, size_t bytes) {
    return ensure_buffer(ctx, ctx->scratch, ctx->scratch_bytes, bytes, "scratch");
}

tnsk_status ensure_twiddles(tnsk_ctx* ctx) {
    if (ctx->d_tw32) return TNSK_OK;
    size_t total32 = 0, total64 = 0;
    for (int l = 0; l <= 16; ++l) {
        size_t M = l > 0 ? ((size_t)1 << (l - 1)) : 1;
        total32 += M * sizeof(float) * 2;
        total64 += M * sizeof(double) * 2;
    }
    std::vector<float> h32;
    std::vector<double> h64;
    h32.reserve(total32 / 4);
    h64.reserve(total64 / 8);
    std::vector<size_t> off32, off64;
    for (int l = 0; l <= 16; ++l) {
        size_t m = (size_t)1 << l;
        size_t M = l > 0 ? m / 2 : 1;
        off32.push_back(h32.size());
        off64.push_back(h64.size());
        for (size_t k = 0; k < M; ++k) {
            // exact argument reduction by symmetry keeps the table within an ulp
            double a = -2.0 * M_PI * (double)k / (double)m;
            double c = std::cos(a), s = std::sin(a);
            h32.push_back((float)c);
            h32.push_back((float)s);
            h64.push_back(c);
            h64.push_back(s);
        }
    }
    void* d32 = nullptr;
    void* d64 = nullptr;
    TNSK_CUDA(cudaMalloc(&d32, h32.size() * sizeof(float)));
    TNSK_CUDA(cudaMalloc(&d64, h64.size() * sizeof(double)));
    TNSK_CUDA(cudaMemcpy(d32, h32.data(), h32.size() * sizeof(float), cudaMemcpyHostToDevice));
    TNSK_CUDA(cudaMemcpy(d64, h64.data(), h64.size() * sizeof(double), cudaMemcpyHostToDevice));
    const void* p32[17];
    const void* p64[17];
    for (int l = 0; l <= 16; ++l) {
        ctx->tw32[l] = (float*)d32 + off32[l];
        ctx->tw64[l] = (double*)d64 + off64[l];
        p32[l] = ctx->tw32[l];
        p64[l] = ctx->tw64[l];
    }
    TNSK_CUDA(cudaMalloc((void**)&ctx->d_tw32, sizeof(p32)));
    TNSK_CUDA(cudaMalloc((void**)&ctx->d_tw64, sizeof(p64)));
    TNSK_CUDA(cudaMemcpy(ctx->d_tw32, p32, sizeof(p32), cudaMemcpyHostToDevice));
    TNSK_CUDA(cudaMemcpy(ctx->d_tw64, p64, sizeof(p64), cudaMemcpyHostToDevice));
    return TNSK_OK;
}

tnsk_status check_ctx(tnsk_ctx* ctx) {
    if (!ctx) return TNSK_ERR_INVALID;
    if (ctx->deferred != TNSK_OK) {
        tnsk_status s = ctx->deferred;
        ctx->deferred = TNSK_OK;
        return s;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return TNSK_OK;
}

}  // namespace

namespace tnsk {
tnsk_status ctx_fail(tnsk_ctx* ctx, tnsk_status st, const std::string& msg) { return fail(ctx, st, msg); }
tnsk_status ctx_cuda_fail(tnsk_ctx* ctx, cudaError_t e, const char* where) { return cuda_fail(ctx, e, where); }
tnsk_status ctx_check(tnsk_ctx* ctx) { return check_ctx(ctx); }
tnsk_status ctx_ensure_scratch(tnsk_ctx* ctx, size_t bytes) { return ensure_scratch(ctx, bytes); }
tnsk_status ctx_ensure_work(tnsk_ctx* ctx, size_t bytes) {
    return ensure_buffer(ctx, ctx->work, ctx->work_bytes, bytes, "work buffer");
}
}  // namespace tnsk

// ---------------------------------------------------------------------------
// Arena: carve typed regions out of the ctx scratch, then upload host staging.
// ---------------------------------------------------------------------------
namespace tnsk {

size_t Arena::take(size_t bytes, size_t align) {
    size_t at = (used + align - 1) / align * align;
    used = at + bytes;
    return at;
}

}  // namespace tnsk

extern "C" {

tnsk_status tnsk_create(tnsk_ctx** out, int device, void* cuda_stream) {
    if (!out) return TNSK_ERR_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return TNSK_ERR_CUDA;
    }
    tnsk_ctx* ctx = new tnsk_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(device) != cudaSuccess || cudaMalloc((void**)&ctx->d_err, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return TNSK_ERR_CUDA;
    }
    if (ensure_twiddles(ctx) != TNSK_OK) {
        delete ctx;
        return TNSK_ERR_CUDA;
    }
    if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();  // no second stream: method 1 and 2 then run in sequence
        if (ctx->side) cudaStreamDestroy(ctx->side);
        if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
        ctx->side = nullptr;
        ctx->ev_fork = ctx->ev_join = nullptr;
    }
    *out = ctx;
    return TNSK_OK;
}

tnsk_status tnsk_destroy(tnsk_ctx* ctx) {
    if (!ctx) return TNSK_ERR_INVALID;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->norm) cudaFree(ctx->norm);
    if (ctx->tw32[0]) cudaFree(ctx->tw32[0]);
    if (ctx->tw64[0]) cudaFree(ctx->tw64[0]);
    if (ctx->d_tw32) cudaFree(ctx->d_tw32);
    if (ctx->d_tw64) cudaFree(ctx->d_tw64);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->aux) cudaFree(ctx->aux);
    if (ctx->work) cudaFree(ctx->work);
    if (ctx->open_buf) cudaFree(ctx->open_buf);
    if (ctx->side) {
        cudaStreamSynchronize(ctx->side);
        cudaStreamDestroy(ctx->side);
        cudaEventDestroy(ctx->ev_fork);
        cudaEventDestroy(ctx->ev_join);
    }
    delete ctx;
    return TNSK_OK;
}

tnsk_status tnsk_set_stream(tnsk_ctx* ctx, void* cuda_stream) {
    if (!ctx) return TNSK_ERR_INVALID;
    ctx->stream = (cudaStream_t)cuda_stream;
    return TNSK_OK;
}

tnsk_status tnsk_sync(tnsk_ctx* ctx) {
    if (!ctx) return TNSK_ERR_INVALID;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    int err = 0;
    e = cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy(err)");
    if (err != DEVERR_NONE) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        if (err == DEVERR_TIMEOUT) return fail(ctx, TNSK_ERR_TIMEOUT, "a device-side wait gave up");
        return fail(ctx, TNSK_ERR_INVALID, "a device-side bounds check failed");
    }
    if (ctx->deferred != TNSK_OK) {
        tnsk_status s = ctx->deferred;
        ctx->deferred = TNSK_OK;
        return s;
    }
    return TNSK_OK;
}

const char* tnsk_status_string(tnsk_status s) {
    switch (s) {
        case TNSK_OK: return "TNSK_OK";
        case TNSK_ERR_INVALID: return "TNSK_ERR_INVALID";
        case TNSK_ERR_CYCLIC: return "TNSK_ERR_CYCLIC";
        case TNSK_ERR_UNSUPPORTED: return "TNSK_ERR_UNSUPPORTED";
        case TNSK_ERR_CUDA: return "TNSK_ERR_CUDA";
        case TNSK_ERR_OOM: return "TNSK_ERR_OOM";
        case TNSK_ERR_TIMEOUT: return "TNSK_ERR_TIMEOUT";
        case TNSK_ERR_UNREACHABLE: return "TNSK_ERR_UNREACHABLE";
    }
    return "TNSK_UNKNOWN";
}

const char* tnsk_last_error(tnsk_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

tnsk_status tnsk_count_sketch(tnsk_ctx* ctx, uint64_t seed, uint64_t rep, uint64_t tid, int64_t n, int64_t m,
                              int32_t* bins, int8_t* signs) {
    tnsk_status st = check_ctx(ctx);
    if (st != TNSK_OK) return st;
    if (n < 0 || m < 1 || m > TNSK_MAX_M || (m & (m - 1)) || (n > 0 && (!bins || !signs)))
        return fail(ctx, TNSK_ERR_INVALID, "count_sketch: need n >= 0, m a power of two <= 65536, buffers");
    TNSK_CUDA(launch_count_sketch(seed, rep, tid, n, m, bins, signs, ctx->stream));
    return TNSK_OK;
}

// Host part of a batch: validation and layout of descriptors and scratch.
static tnsk_status build_plan(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, const tnsk_params* params,
                              double* const* outs, double* const* per_reps, bool sketch_only, BatchPlan& plan,
                              bool& fp64, bool zero_ok = false, const NormBatch* nb = nullptr,
                              const tnsk_schedule* sched = nullptr, const int64_t* rep_stride = nullptr) {
    if (B < 0 || (B > 0 && (!nets || !params))) return fail(ctx, TNSK_ERR_INVALID, "null batch arguments");
    std::vector<NetInfo> infos(B);
    for (int b = 0; b < B; ++b) {
        std::string why;
        const char* diag = nb && !nb->diag.empty() && !nb->diag[b].empty() ? nb->diag[b].data() : nullptr;
        tnsk_status st = validate(nets[b], params[b], infos[b], why, zero_ok, diag);
        if (st != TNSK_OK) return fail(ctx, st, "network " + std::to_string(b) + ": " + why);
        if (!sketch_only && (!outs || !outs[b])) return fail(ctx, TNSK_ERR_INVALID, "null output buffer");
    }
    // precision of the whole batch: one kind per launch sequence
    fp64 = B > 0 && params[0].prec == TNSK_PREC_FP64;
    for (int b = 1; b < B; ++b)
        if ((params[b].prec == TNSK_PREC_FP64) != fp64)
            return fail(ctx, TNSK_ERR_UNSUPPORTED, "mixed precisions in one batch");
    return plan_batch(infos, nets, params, outs, per_reps, fp64, sketch_only, plan, ctx->last_error, sched,
                      rep_stride);
}

// Device part: the launch sequence of a planned batch whose descriptors are
// already at base + plan.desc_off.
// The normalisation launch of a batch (WLOG 2 / 3 rewrite of acyclic networks), if any.
struct NormRun {
    const NormJob* d_jobs = nullptr;
    int n = 0;
    int64_t most = 0;
};

static tnsk_status launch_plan(tnsk_ctx* ctx, const BatchPlan& plan, unsigned char* base, bool fp64,
                               void* sketch_out, const NormRun& nr = NormRun{}, tnsk_pairs* prelude = nullptr) {
    cudaStream_t s = ctx->stream;
    if (nr.n) {  // the rewritten tensors first: method 2 reads them
        ctx->prof.begin(TNSK_K_NORMALIZE, s);
        TNSK_CUDA(launch_normalize(nr.d_jobs, nr.n, nr.most, s));
        ctx->prof.end(s);
    }
    if (plan.zero_bytes) TNSK_CUDA(cudaMemsetAsync(base + plan.zero_off, 0, plan.zero_bytes, s));
    if (sketch_out && plan.sketch_user_bytes) TNSK_CUDA(cudaMemsetAsync(sketch_out, 0, plan.sketch_user_bytes, s));
    Profiler& pf = ctx->prof;
    if (plan.n_reqs) {
        pf.begin(TNSK_K_TABLES, s);
        TNSK_CUDA(launch_draw_tables((const TabReq*)(base + plan.reqs_off), plan.n_reqs, plan.n_table_rows,
                                     (uint32_t*)(base + plan.tabs_off), s));
        pf.end(s);
    }
    // Methods 1 and 2 share only the tables: with both in the batch (and per-kernel
    // timing off), method 1 runs on the ctx's second stream while method 2 runs on
    // the ctx stream, joined before the combine. Inside a stream capture the fork and
    // join become graph edges.
    const bool fork = !pf.on && ctx->side && plan.m1.n_nets && plan.m2.n_nets && !sketch_out;
    cudaStream_t s1 = s;
    if (fork) {
        TNSK_CUDA(cudaEventRecord(ctx->ev_fork, s));
        TNSK_CUDA(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
        s1 = ctx->side;
    }
    tnsk_status st = TNSK_OK;
    if (plan.m1.n_nets) {
        void* xs = sketch_out ? sketch_out : (void*)(base + plan.m1.xs_off);
        pf.begin(TNSK_K_M1_SCATTER, s1);
        cudaError_t e = launch_m1_scatters(plan, base, xs, fp64, s1);
        if (e == cudaSuccess) e = launch_m1_diag(plan, base, xs, fp64, s1);  // WLOG 1 copy tensors
        pf.end(s1);
        if (e == cudaSuccess && !sketch_out) {
            pf.begin(TNSK_K_M1_SPECTRUM, s1);
            e = launch_m1_spectra(plan, base, xs,
                                  fp64 ? (const void* const*)ctx->d_tw64 : (const void* const*)ctx->d_tw32, fp64,
                                  s1);
            pf.end(s1);
        }
        if (e != cudaSuccess) st = cuda_fail(ctx, e, "method 1 launch");
    }
    if (fork) {  // joined on every path, so a capture never ends with the side stream open
        const cudaError_t e1 = cudaEventRecord(ctx->ev_join, ctx->side);
        if (st == TNSK_OK && e1 != cudaSuccess) st = cuda_fail(ctx, e1, "cudaEventRecord");
    }
    // the plan's prelude (tnsk_plan_set_prelude): pair contractions that feed method 2,
    // on the ctx stream, so they overlap method 1 on the second stream
    if (st == TNSK_OK && prelude && !sketch_out) st = tnsk_pairs_run(ctx, prelude);
    if (st == TNSK_OK && plan.m2.n_nets && !sketch_out) {
        st = run_method2(plan, base, fp64, fp64 ? (const void* const*)ctx->d_tw64 : (const void* const*)ctx->d_tw32, s,
                         pf, ctx->d_err, ctx->last_error, ctx->inject);
        ctx->inject = 0;  // one-shot
    }
    if (fork) {
        const cudaError_t e2 = cudaStreamWaitEvent(s, ctx->ev_join, 0);
        if (st == TNSK_OK && e2 != cudaSuccess) st = cuda_fail(ctx, e2, "cudaStreamWaitEvent");
    }
    if (st != TNSK_OK) return st;
    if (!sketch_out && plan.n_comb) {
        pf.begin(TNSK_K_COMBINE, s);
        TNSK_CUDA(launch_combine((const CombineItem*)(base + plan.comb_off), plan.n_comb,
                                 (const double*)(base + plan.yrep_off), s));
        pf.end(s);
    }
    return TNSK_OK;
}

// Batch driver shared by tnsk_estimate, tnsk_estimate_batch and tnsk_m1_sketch.
static tnsk_status run_batch_core(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, const tnsk_params* params,
                                  double* const* outs, double* const* per_reps, void* sketch_out,
                                  size_t* yrep_off = nullptr, int64_t* yrep_n = nullptr,
                                  const int64_t* rep_stride = nullptr) {
    tnsk_status st = check_ctx(ctx);
    if (st != TNSK_OK) return st;
    if (B == 0) return TNSK_OK;
    // acyclic networks with traces or repeated contractions are rewritten first
    NormBatch nb;
    std::string why;
    st = normalize_batch(B, nets, params, nb, why);
    if (st != TNSK_OK) return fail(ctx, st, why);
    if (!nb.jobs.empty()) {
        st = ensure_buffer(ctx, ctx->norm, ctx->norm_bytes, nb.bytes, "normalisation buffer");
        if (st != TNSK_OK) return st;
        normalize_bind(nb, ctx->norm);
    }
    BatchPlan plan;
    bool fp64 = false;
    st = build_plan(ctx, B, nb.used ? nb.view.data() : nets, params, outs, per_reps, sketch_out != nullptr, plan,
                    fp64, false, &nb, nullptr, rep_stride);
    if (st != TNSK_OK) return st;
    st = ensure_scratch(ctx, plan.arena.used);
    if (st != TNSK_OK) return st;
    st = finalize_plan(plan, ctx->scratch, ctx->last_error);
    if (st != TNSK_OK) return st;
    // descriptors (pageable host staging: the copy is complete on return)
    if (!plan.host_desc.empty())
        TNSK_CUDA(cudaMemcpyAsync(ctx->scratch + plan.desc_off, plan.host_desc.data(), plan.host_desc.size(),
                                  cudaMemcpyHostToDevice, ctx->stream));
    recycle_host_desc(plan.host_desc);  // a pageable source is consumed when the call returns
    NormRun nr;
    if (!nb.jobs.empty()) {
        TNSK_CUDA(cudaMemcpyAsync(ctx->norm + nb.desc_off, nb.jobs.data(), nb.jobs.size() * sizeof(NormJob),
                                  cudaMemcpyHostToDevice, ctx->stream));
        nr = NormRun{(const NormJob*)(ctx->norm + nb.desc_off), (int)nb.jobs.size(), nb.most};
    }
    if (yrep_off) *yrep_off = plan.yrep_off;
    if (yrep_n) *yrep_n = plan.yrep_n;
    return launch_plan(ctx, plan, ctx->scratch, fp64, sketch_out, nr);
}

// Method 2 with open legs (Corollary "full-to-partial-tc"): every output entry of a
// TNSK_ACYCLIC network with open modes is the full estimate of the network whose
// tensors are sliced at that entry's open indices. Each tensor with open modes is
// written once, its open modes first (in the output order) and its other modes after
// them in their order, so that every slice is a contiguous block; the entries then run
// as networks of their own in one batch, with the same hash functions (the edges keep
// their order) and the per-rep values of entry o at per_rep[r O + o]. Other networks
// of the batch pass through. Networks whose structure does not check out here pass
// through unchanged and are reported by the planner.
namespace {
struct OpenExpansion {
    std::vector<tnsk_network> nets;
    std::vector<tnsk_params> params;
    std::vector<double*> outs, reps;
    std::vector<int64_t> stride;
    std::vector<std::vector<tnsk_tensor>> X;            // per expanded entry
    std::vector<std::vector<std::vector<int64_t>>> dims;  // per source network: sliced dims per tensor
    std::vector<std::vector<int32_t>> edges;             // per source network: renumbered edges
    std::vector<NormJob> jobs;
    std::vector<size_t> off;  // per job: output offset in the buffer
    std::vector<std::pair<size_t, int>> sliced;  // (entry, tensor) whose data is an offset into the buffer
    size_t bytes = 0;
    int64_t most = 0;
};
constexpr int64_t kMaxOpenEntries = 1 << 16;  // expanded entries per call
}  // namespace

static tnsk_status expand_open_m2(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, const tnsk_params* params,
                                  double* const* outs, double* const* per_reps, OpenExpansion& E) {
    int64_t entries = 0;
    E.dims.resize(B);
    E.edges.resize(B);
    // first pass: which networks expand, their jobs and buffer size
    struct Src {
        bool expand = false;
        int64_t O = 1;
        std::vector<int> mode_off, open_pos, new_id, job;
        std::vector<int64_t> slice;  // per tensor: entries per slice (its non-open modes)
        std::vector<std::vector<int>> opens;  // per tensor: its open modes in output order
    };
    std::vector<Src> src(B);
    for (int b = 0; b < B; ++b) {
        const tnsk_network& N = nets[b];
        Src& S = src[b];
        if (params[b].method != TNSK_ACYCLIC || N.n_open <= 0 || N.p < 1 || !N.X || !N.open || N.t < 0 ||
            (N.t > 0 && !N.edges))
            continue;
        // structure: modes, contracted modes, the open list a permutation of the rest
        S.mode_off.assign(N.p + 1, 0);
        bool ok = true;
        for (int k = 0; k < N.p && ok; ++k) {
            const tnsk_tensor& T = N.X[k];
            ok = T.order >= 0 && T.order <= TNSK_MAX_ORDER && (T.order == 0 || T.dims) && (T.rung || T.data);
            int64_t numel = 1;  // dims non-negative, at most 2^40 entries (else the planner reports it)
            for (int d = 0; d < T.order && ok; ++d) {
                ok = T.dims[d] >= 0 && (T.dims[d] == 0 || numel <= ((int64_t)1 << 40) / T.dims[d]);
                if (ok) numel *= T.dims[d];
            }
            S.mode_off[k + 1] = S.mode_off[k] + (ok ? T.order : 0);
        }
        const int q = S.mode_off[N.p];
        std::vector<int> tensor_of(q), used(q, 0);
        for (int k = 0; k < N.p && ok; ++k)
            for (int g = S.mode_off[k]; g < S.mode_off[k + 1]; ++g) tensor_of[g] = k;
        for (int e = 0; e < N.t && ok; ++e)
            for (int side = 0; side < 2 && ok; ++side) {
                const int g = N.edges[2 * e + side];
                ok = g >= 0 && g < q && !used[g];
                if (ok) used[g] = 1;
            }
        S.open_pos.assign(q, -1);
        for (int j = 0; j < N.n_open && ok; ++j) {
            const int g = N.open[j];
            ok = g >= 0 && g < q && !used[g] && S.open_pos[g] < 0;
            if (ok) S.open_pos[g] = j;
        }
        for (int g = 0; g < q && ok; ++g) ok = used[g] || S.open_pos[g] >= 0;
        if (!ok) continue;
        auto dim_of = [&](int g) { return N.X[tensor_of[g]].dims[g - S.mode_off[tensor_of[g]]]; };
        for (int j = 0; j < N.n_open; ++j)  // (capped just above the limit: no overflow)
            S.O = std::min<int64_t>(S.O * dim_of(N.open[j]), kMaxOpenEntries + 1);
        entries += S.O;
        if (S.O == 0 || entries > kMaxOpenEntries)
            return fail(ctx, TNSK_ERR_UNSUPPORTED,
                        "network " + std::to_string(b) + ": method 2 with open legs takes up to 2^16 output entries "
                        "per call (one full estimate each), and none of an empty output");
        S.expand = true;
        // renumbered contracted modes and edges; per tensor its open modes (output order)
        S.new_id.assign(q, -1);
        int nid = 0;
        for (int g = 0; g < q; ++g)
            if (S.open_pos[g] < 0) S.new_id[g] = nid++;
        E.edges[b].resize(2 * (size_t)N.t);
        for (int e = 0; e < 2 * N.t; ++e) E.edges[b][e] = S.new_id[N.edges[e]];
        S.opens.assign(N.p, {});
        S.slice.assign(N.p, 1);
        S.job.assign(N.p, -1);
        E.dims[b].assign(N.p, {});
        for (int j = 0; j < N.n_open; ++j) S.opens[tensor_of[N.open[j]]].push_back(N.open[j]);
        for (int k = 0; k < N.p; ++k)
            if (N.X[k].rung && !S.opens[k].empty())
                return fail(ctx, TNSK_ERR_UNSUPPORTED,
                            "network " + std::to_string(b) + ": a grouped tensor with open modes (method 2)");
        for (int k = 0; k < N.p; ++k) {
            const tnsk_tensor& T = N.X[k];
            for (int d = 0; d < T.order; ++d)
                if (S.open_pos[S.mode_off[k] + d] < 0) {
                    E.dims[b][k].push_back(T.dims[d]);
                    S.slice[k] *= T.dims[d];
                }
            if (S.opens[k].empty()) continue;
            // the tensor with its open modes first: a strided gather (normalize_kernel)
            NormJob J{};
            J.src = T.data;
            J.src_dtype = T.dtype;
            J.dst_f64 = T.dtype == TNSK_F64;
            int64_t str[TNSK_MAX_ORDER], st = 1;
            for (int d = T.order - 1; d >= 0; --d) str[d] = st, st *= T.dims[d];
            J.numel = st;
            J.n = 0;
            for (int g : S.opens[k]) {
                J.dim[J.n] = dim_of(g);
                J.str[J.n++] = str[g - S.mode_off[k]];
            }
            for (int d = 0; d < T.order; ++d)
                if (S.open_pos[S.mode_off[k] + d] < 0) {
                    J.dim[J.n] = T.dims[d];
                    J.str[J.n++] = str[d];
                }
            J.nd = 0;
            S.job[k] = (int)E.jobs.size();
            E.bytes = (E.bytes + 255) & ~(size_t)255;
            E.off.push_back(E.bytes);
            E.bytes += (size_t)J.numel * (J.dst_f64 ? 8 : 4);
            E.most = std::max(E.most, J.numel);
            E.jobs.push_back(J);
        }
    }
    if (E.jobs.empty() && entries == 0) return TNSK_OK;
    // the expanded batch
    E.nets.reserve(B + entries);
    E.X.reserve(entries);
    for (int b = 0; b < B; ++b) {
        const Src& S = src[b];
        if (!S.expand) {
            E.nets.push_back(nets[b]);
            E.params.push_back(params[b]);
            E.outs.push_back(outs ? outs[b] : nullptr);
            E.reps.push_back(per_reps ? per_reps[b] : nullptr);
            E.stride.push_back(0);
            continue;
        }
        const tnsk_network& N = nets[b];
        for (int64_t o = 0; o < S.O; ++o) {
            E.X.emplace_back(N.X, N.X + N.p);
            std::vector<tnsk_tensor>& X = E.X.back();
            for (int k = 0; k < N.p; ++k) {
                X[k].order = (int32_t)E.dims[b][k].size();
                X[k].dims = E.dims[b][k].data();
                if (S.job[k] < 0) continue;
                // the slice at this entry's indices of the tensor's open modes (row-major
                // over them in output order, the open list's first mode slowest)
                int64_t at = 0;
                for (int g : S.opens[k]) {
                    int64_t stride_o = 1;
                    for (int j = S.open_pos[g] + 1; j < N.n_open; ++j) {
                        const int h = N.open[j];
                        int kk = 0;
                        while (S.mode_off[kk + 1] <= h) ++kk;
                        stride_o *= N.X[kk].dims[h - S.mode_off[kk]];
                    }
                    int kk = 0;
                    while (S.mode_off[kk + 1] <= g) ++kk;
                    const int64_t dg = N.X[kk].dims[g - S.mode_off[kk]];
                    at = at * dg + (o / stride_o) % dg;
                }
                const NormJob& J = E.jobs[S.job[k]];
                // an offset into the buffer until its address is known (run_batch)
                X[k].data = (const void*)(uintptr_t)(E.off[S.job[k]] + (size_t)(at * S.slice[k]) * (J.dst_f64 ? 8 : 4));
                X[k].dtype = J.dst_f64 ? TNSK_F64 : TNSK_F32;
                E.sliced.emplace_back(E.X.size() - 1, k);
            }
            tnsk_network n{};
            n.p = N.p;
            n.X = X.data();
            n.t = N.t;
            n.edges = E.edges[b].data();
            n.n_open = 0;
            n.open = nullptr;
            E.nets.push_back(n);
            E.params.push_back(params[b]);
            E.outs.push_back(outs && outs[b] ? outs[b] + o : nullptr);
            E.reps.push_back(per_reps && per_reps[b] ? per_reps[b] + o : nullptr);
            E.stride.push_back(S.O);
        }
    }
    return TNSK_OK;
}

// Batch driver shared by tnsk_estimate, tnsk_estimate_batch and tnsk_m1_sketch.
static tnsk_status run_batch(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, const tnsk_params* params,
                             double* const* outs, double* const* per_reps, void* sketch_out,
                             size_t* yrep_off = nullptr, int64_t* yrep_n = nullptr) {
    tnsk_status st = check_ctx(ctx);
    if (st != TNSK_OK) return st;
    if (B <= 0 || !nets || !params || sketch_out)
        return run_batch_core(ctx, B, nets, params, outs, per_reps, sketch_out, yrep_off, yrep_n);
    OpenExpansion E;
    st = expand_open_m2(ctx, B, nets, params, outs, per_reps, E);
    if (st != TNSK_OK) return st;
    if (E.nets.empty()) return run_batch_core(ctx, B, nets, params, outs, per_reps, sketch_out, yrep_off, yrep_n);
    // the sliced copies, then the expanded batch on the same stream
    st = ensure_buffer(ctx, ctx->open_buf, ctx->open_bytes,
                       ((E.bytes + 255) & ~(size_t)255) + E.jobs.size() * sizeof(NormJob), "open-leg buffer");
    if (st != TNSK_OK) return st;
    for (size_t j = 0; j < E.jobs.size(); ++j) E.jobs[j].dst = ctx->open_buf + E.off[j];
    for (const auto& sk : E.sliced) {  // the slices' offsets become addresses
        tnsk_tensor& T = E.X[sk.first][sk.second];
        T.data = ctx->open_buf + (uintptr_t)T.data;
    }
    const size_t desc = (E.bytes + 255) & ~(size_t)255;
    if (!E.jobs.empty()) {
        TNSK_CUDA(cudaMemcpyAsync(ctx->open_buf + desc, E.jobs.data(), E.jobs.size() * sizeof(NormJob),
                                  cudaMemcpyHostToDevice, ctx->stream));
        ctx->prof.begin(TNSK_K_NORMALIZE, ctx->stream);
        TNSK_CUDA(launch_normalize((const NormJob*)(ctx->open_buf + desc), (int)E.jobs.size(), E.most, ctx->stream));
        ctx->prof.end(ctx->stream);
    }
    return run_batch_core(ctx, (int32_t)E.nets.size(), E.nets.data(), E.params.data(), E.outs.data(), E.reps.data(),
                          nullptr, yrep_off, yrep_n, E.stride.data());
}

// TNSK_PREC_AUTO (tnsk.h): the FP32 path with the per-rep magnitude sums, the FP64 path
// for the smallest range of reps holding every flagged one, then the combination.
static tnsk_status estimate_auto(tnsk_ctx* ctx, const tnsk_network* net, const tnsk_params* params, double* out,
                                 double* per_rep) {
    tnsk_status st = check_ctx(ctx);
    if (st != TNSK_OK) return st;
    if (params->method != TNSK_GENERAL || net->n_open != 0)
        return fail(ctx, TNSK_ERR_UNSUPPORTED, "TNSK_PREC_AUTO: method 1 (TNSK_GENERAL) without open legs only");
    if (!out) return fail(ctx, TNSK_ERR_INVALID, "null output buffer");
    const int32_t R = params->reps;
    if (R < 1 || R > 65536) return fail(ctx, TNSK_ERR_INVALID, "reps must be in [1, 65536]");
    // per-rep values: the caller's buffer, else the ctx's; one more double for the FP64
    // pass's combined value, which is not used
    const size_t need = (size_t)(R + 1) * sizeof(double);
    unsigned char* auxb = (unsigned char*)ctx->aux;
    st = ensure_buffer(ctx, auxb, ctx->aux_bytes, need, "TNSK_PREC_AUTO buffer");
    ctx->aux = (double*)auxb;
    if (st != TNSK_OK) return st;
    double* yr = per_rep ? per_rep : ctx->aux + 1;
    tnsk_params q = *params;
    q.prec = TNSK_PREC_FP32;
    size_t yoff = 0;
    int64_t yn = 0;
    st = run_batch(ctx, 1, net, &q, &out, &yr, nullptr, &yoff, &yn);
    if (st != TNSK_OK) return st;
    // a one-network plan: its estimates are yrep[0 .. R), the magnitude sums yrep[yn ..)
    std::vector<double> y(R), a(R);
    TNSK_CUDA(cudaMemcpyAsync(y.data(), ctx->scratch + yoff, R * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    TNSK_CUDA(cudaMemcpyAsync(a.data(), ctx->scratch + yoff + (size_t)yn * sizeof(double), R * sizeof(double),
                              cudaMemcpyDeviceToHost, ctx->stream));
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "TNSK_PREC_AUTO");
    const double lg = std::log2((double)std::max<int64_t>(params->m, 1));
    const double c32 = (net->p + 2.0 * lg + 8.0) * std::ldexp(1.0, -24);
    const double c64 = (net->p + 2.0 * lg + 8.0) * std::ldexp(1.0, -53);
    const double tau = std::ldexp(1.0, -17);  // ~7.6e-6 of the rep's own value
    int32_t lo = R, hi = -1;
    for (int32_t r = 0; r < R; ++r)
        if (c32 * a[r] > tau * std::fabs(y[r])) {
            lo = std::min(lo, r);
            hi = r;
        }
    if (hi >= lo) {
        tnsk_params q64 = *params;
        q64.prec = TNSK_PREC_FP64;
        q64.rep0 = params->rep0 + lo;
        q64.reps = hi - lo + 1;
        q64.groups = 1;
        double* o64 = ctx->aux;
        double* p64 = yr + lo;
        st = run_batch(ctx, 1, net, &q64, &o64, &p64, nullptr);
        if (st != TNSK_OK) return st;
        TNSK_CUDA(cudaMemcpyAsync(y.data() + lo, p64, (size_t)(hi - lo + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                                  ctx->stream));
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "TNSK_PREC_AUTO");
        st = tnsk_combine(ctx, R, 1, yr, params->groups, out);
        if (st != TNSK_OK) return st;
    }
    double worst = 0.0;
    for (int32_t r = 0; r < R; ++r) {
        const double c = (r >= lo && r <= hi) ? c64 : c32;
        const double b = a[r] > 0.0 ? c * a[r] / std::fabs(y[r]) : 0.0;  // +inf when y_r = 0 < A_r
        worst = std::max(worst, b);
    }
    ctx->auto_fp64_reps = hi >= lo ? hi - lo + 1 : 0;
    ctx->auto_max_bound = worst;
    return TNSK_OK;
}

struct tnsk_plan {
    BatchPlan plan;
    tnsk_pairs* prelude = nullptr;  // run ahead of method 2 in every run (tnsk_plan_set_prelude)
    bool fp64 = false;
    int device = 0;
    unsigned char* dev = nullptr;  // descriptors + scratch of this plan
    NormBatch norm;                   // rewritten acyclic networks (WLOG 2 / 3), if any
    unsigned char* norm_dev = nullptr;  // their tensors and descriptors
    NormRun nr;
    int64_t runs = 0;
    cudaGraphExec_t graph = nullptr;  // the launch sequence, captured on the second run
    bool no_graph = false;            // capture failed or is not possible: launch directly
};

tnsk_status tnsk_debug_inject(tnsk_ctx* ctx, int32_t what) {
    if (!ctx || what < 0 || what > 1) return TNSK_ERR_INVALID;
    ctx->inject = what;
    return TNSK_OK;
}

tnsk_status tnsk_profile(tnsk_ctx* ctx, int32_t enable) {
    if (!ctx) return TNSK_ERR_INVALID;
    ctx->prof.on = enable != 0;
    return TNSK_OK;
}

tnsk_status tnsk_profile_read(tnsk_ctx* ctx, double* ms, int64_t* launches) {
    if (!ctx || !ms || !launches) return TNSK_ERR_INVALID;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    for (int k = 0; k < TNSK_KERNEL_KINDS; ++k) {
        ms[k] = 0;
        launches[k] = 0;
    }
    for (auto& r : ctx->prof.recs) {
        float t = 0;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess && r.kind >= 0 && r.kind < TNSK_KERNEL_KINDS) {
            ms[r.kind] += t;
            launches[r.kind] += 1;
        }
        ctx->prof.pool.push_back(r.a);
        ctx->prof.pool.push_back(r.b);
    }
    ctx->prof.recs.clear();
    cudaGetLastError();
    return TNSK_OK;
}

static tnsk_status create_plan(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, const tnsk_params* params,
                               double* const* outs, double* const* per_reps, bool zero_ok, tnsk_plan** out,
                               const tnsk_schedule* sched = nullptr) {
    if (!out) return TNSK_ERR_INVALID;
    *out = nullptr;
    tnsk_status st = check_ctx(ctx);
    if (st != TNSK_OK) return st;
    tnsk_plan* p = new tnsk_plan();
    p->device = ctx->device;
    auto drop = [&]() {
        cudaFree(p->dev);
        cudaFree(p->norm_dev);
        delete p;
    };
    std::string why;
    st = normalize_batch(B, nets, params, p->norm, why);
    if (st != TNSK_OK) {
        drop();
        return fail(ctx, st, why);
    }
    cudaError_t e = cudaSuccess;
    if (!p->norm.jobs.empty()) {
        if (cudaMalloc((void**)&p->norm_dev, p->norm.bytes) != cudaSuccess) {
            cudaGetLastError();
            p->norm_dev = nullptr;
            drop();
            return fail(ctx, TNSK_ERR_OOM, "plan normalisation buffer allocation failed");
        }
        normalize_bind(p->norm, p->norm_dev);
        e = cudaMemcpy(p->norm_dev + p->norm.desc_off, p->norm.jobs.data(), p->norm.jobs.size() * sizeof(NormJob),
                       cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            drop();
            return cuda_fail(ctx, e, "cudaMemcpy(normalisation descriptors)");
        }
        p->nr = NormRun{(const NormJob*)(p->norm_dev + p->norm.desc_off), (int)p->norm.jobs.size(), p->norm.most};
    }
    st = build_plan(ctx, B, p->norm.used ? p->norm.view.data() : nets, params, outs, per_reps, false, p->plan,
                    p->fp64, zero_ok, &p->norm, sched);
    if (st != TNSK_OK) {
        drop();
        return st;
    }
    if (cudaMalloc((void**)&p->dev, std::max<size_t>(p->plan.arena.used, 256)) != cudaSuccess) {
        cudaGetLastError();
        p->dev = nullptr;
        drop();
        return fail(ctx, TNSK_ERR_OOM, "plan scratch allocation failed");
    }
    st = finalize_plan(p->plan, p->dev, ctx->last_error);
    if (st != TNSK_OK) {
        drop();
        return st;
    }
    if (!p->plan.host_desc.empty())
        e = cudaMemcpy(p->dev + p->plan.desc_off, p->plan.host_desc.data(), p->plan.host_desc.size(),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        drop();
        return cuda_fail(ctx, e, "cudaMemcpy(plan descriptors)");
    }
    recycle_host_desc(p->plan.host_desc);
    *out = p;
    return TNSK_OK;
}

tnsk_status tnsk_plan_create(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, const tnsk_params* params,
                             double* const* outs, double* const* per_reps, tnsk_plan** out) {
    return create_plan(ctx, B, nets, params, outs, per_reps, false, out);
}

tnsk_status tnsk_plan_create_scheduled(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets,
                                       const tnsk_params* params, double* const* outs, double* const* per_reps,
                                       const tnsk_schedule* sched, tnsk_plan** out) {
    return create_plan(ctx, B, nets, params, outs, per_reps, false, out, sched);
}

// The scatter autotuner (tnsk.h): every candidate schedule planned on the host and
// laid out in the ctx scratch; per scatter list the launch is timed alone.
tnsk_status tnsk_autotune(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, const tnsk_params* params,
                          int32_t trials, tnsk_schedule* sched, double* ms_default, double* ms_tuned) {
    tnsk_status st = check_ctx(ctx);
    if (st != TNSK_OK) return st;
    if (!sched || trials < 1 || trials > 64) return fail(ctx, TNSK_ERR_INVALID, "autotune: arguments");
    constexpr int L = TNSK_SCATTER_LISTS;
    static const int kCaps[] = {8, 16, 32}, kScales[] = {1, 2, 4};
    struct Cand {
        int cap, scale;
    };
    std::vector<Cand> cands;
    for (int c : kCaps)
        for (int s : kScales) cands.push_back({c, s});
    NormBatch nb;
    std::string why;
    st = normalize_batch(B, nets, params, nb, why);
    if (st != TNSK_OK) return fail(ctx, st, why);
    if (!nb.jobs.empty()) {
        st = ensure_buffer(ctx, ctx->norm, ctx->norm_bytes, nb.bytes, "normalisation buffer");
        if (st != TNSK_OK) return st;
        normalize_bind(nb, ctx->norm);
    }
    const tnsk_network* view = nb.used ? nb.view.data() : nets;
    // outputs are not written (only the scatter runs); the planner wants non-null ones
    std::vector<double*> outs(B, nullptr);
    double dummy = 0.0;
    for (int b = 0; b < B; ++b) outs[b] = &dummy;
    std::vector<std::vector<double>> ms(cands.size() + 1, std::vector<double>(L, 0.0));
    std::vector<std::vector<int>> cnt(cands.size() + 1, std::vector<int>(L, 0));
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return cuda_fail(ctx, cudaGetLastError(), "autotune events");
    auto done = [&](tnsk_status s) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return s;
    };
    for (size_t ci = 0; ci <= cands.size(); ++ci) {  // the last entry: the default schedule
        tnsk_schedule cs{};
        if (ci < cands.size())
            for (int l = 0; l < L; ++l) {
                cs.rep_cap[l] = cands[ci].cap;
                cs.chunk_scale[l] = cands[ci].scale;
            }
        BatchPlan plan;
        bool fp64 = false;
        st = build_plan(ctx, B, view, params, outs.data(), nullptr, false, plan, fp64, false, &nb,
                        ci < cands.size() ? &cs : nullptr);
        if (st != TNSK_OK) return done(st);
        st = ensure_scratch(ctx, plan.arena.used);
        if (st != TNSK_OK) return done(st);
        unsigned char* base = ctx->scratch;
        st = finalize_plan(plan, base, ctx->last_error);
        if (st != TNSK_OK) return done(st);
        if (!plan.host_desc.empty() &&
            cudaMemcpyAsync(base + plan.desc_off, plan.host_desc.data(), plan.host_desc.size(), cudaMemcpyHostToDevice,
                            ctx->stream) != cudaSuccess)
            return done(cuda_fail(ctx, cudaGetLastError(), "autotune descriptors"));
        if (plan.zero_bytes && cudaMemsetAsync(base + plan.zero_off, 0, plan.zero_bytes, ctx->stream) != cudaSuccess)
            return done(cuda_fail(ctx, cudaGetLastError(), "autotune memset"));
        if (plan.n_reqs &&
            launch_draw_tables((const TabReq*)(base + plan.reqs_off), plan.n_reqs, plan.n_table_rows,
                               (uint32_t*)(base + plan.tabs_off), ctx->stream) != cudaSuccess)
            return done(cuda_fail(ctx, cudaGetLastError(), "autotune tables"));
        void* xs = base + plan.m1.xs_off;
        for (int l = 0; l < L; ++l) {
            cnt[ci][l] = plan.m1.work_count[l];
            if (!plan.m1.work_count[l]) continue;
            // one untimed launch, then `trials` timed ones
            cudaError_t e = launch_m1_scatter_list(plan, base, xs, fp64, l, ctx->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
            for (int t = 0; t < trials && e == cudaSuccess; ++t)
                e = launch_m1_scatter_list(plan, base, xs, fp64, l, ctx->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e != cudaSuccess) return done(cuda_fail(ctx, e, "autotune launch"));
            ms[ci][l] = (double)t / trials;
        }
    }
    // per list, the fastest candidate (a list a candidate leaves empty moved its work to
    // another list, so such candidates are compared on the list sums of every list)
    *sched = tnsk_schedule{};
    const size_t def = cands.size();
    double tot_def = 0.0, tot_best = 0.0;
    for (int l = 0; l < L; ++l) tot_def += ms[def][l];
    for (int l = 0; l < L; ++l) {
        if (!cnt[def][l]) continue;
        size_t best = def;
        for (size_t ci = 0; ci < cands.size(); ++ci)
            if (cnt[ci][l] && ms[ci][l] < ms[best][l]) best = ci;
        tot_best += ms[best][l];
        if (best != def) {
            sched->rep_cap[l] = cands[best].cap;
            sched->chunk_scale[l] = cands[best].scale;
        }
    }
    if (ms_default) *ms_default = tot_def;
    if (ms_tuned) *ms_tuned = tot_best;
    return done(TNSK_OK);
}

tnsk_status tnsk_plan_run(tnsk_ctx* ctx, tnsk_plan* plan) {
    if (!plan) return TNSK_ERR_INVALID;
    tnsk_status st = check_ctx(ctx);
    if (st != TNSK_OK) return st;
    if (ctx->device != plan->device) return fail(ctx, TNSK_ERR_INVALID, "plan made on another device");
    cudaStream_t s = ctx->stream;
    // the first run launches directly (and sets every kernel attribute); later runs
    // replay one CUDA graph of the same sequence (not on the legacy stream, whose
    // work cannot be captured, and not while per-kernel timing is on)
    if (plan->runs++ >= 1 && !ctx->prof.on && !plan->no_graph && s != nullptr) {
        if (!plan->graph) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            tnsk_status st = TNSK_ERR_CUDA;
            if (e == cudaSuccess) {
                st = launch_plan(ctx, plan->plan, plan->dev, plan->fp64, nullptr, plan->nr, plan->prelude);
                e = cudaStreamEndCapture(s, &g);
            }
            if (e == cudaSuccess && st == TNSK_OK && g) e = cudaGraphInstantiate(&plan->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess || st != TNSK_OK || !plan->graph) {
                cudaGetLastError();
                plan->graph = nullptr;
                plan->no_graph = true;
                ctx->last_error.clear();
            }
        }
        if (plan->graph) {
            cudaError_t e = cudaGraphLaunch(plan->graph, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
            return TNSK_OK;
        }
    }
    return launch_plan(ctx, plan->plan, plan->dev, plan->fp64, nullptr, plan->nr, plan->prelude);
}

tnsk_status tnsk_plan_set_prelude(tnsk_ctx* ctx, tnsk_plan* plan, tnsk_pairs* pairs) {
    if (!plan) return TNSK_ERR_INVALID;
    tnsk_status st = check_ctx(ctx);
    if (st != TNSK_OK) return st;
    if (ctx->device != plan->device) return fail(ctx, TNSK_ERR_INVALID, "plan made on another device");
    plan->prelude = pairs;
    if (plan->graph) {  // the captured sequence changes: capture again on the next run
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
        cudaGraphExecDestroy(plan->graph);
        plan->graph = nullptr;
    }
    return TNSK_OK;
}

tnsk_status tnsk_plan_destroy(tnsk_plan* plan) {
    if (!plan) return TNSK_ERR_INVALID;
    cudaSetDevice(plan->device);
    cudaDeviceSynchronize();
    if (plan->graph) cudaGraphExecDestroy(plan->graph);
    cudaFree(plan->dev);
    cudaFree(plan->norm_dev);
    delete plan;
    return TNSK_OK;
}

// ---------------------------------------------------------------------------
// Turnstile streams (Sec. 4.2): one method-1 network whose sketches stay in a plan's
// memory; updates change them in place, estimates rerun the transform, product and
// combination on them.
// ---------------------------------------------------------------------------
struct tnsk_stream {
    tnsk_plan* plan = nullptr;
};

tnsk_status tnsk_stream_create(tnsk_ctx* ctx, const tnsk_network* net, const tnsk_params* params, double* out,
                               double* per_rep, tnsk_stream** out_stream) {
    if (!out_stream) return TNSK_ERR_INVALID;
    *out_stream = nullptr;
    tnsk_status st = check_ctx(ctx);
    if (st != TNSK_OK) return st;
    if (!net || !params || !out) return fail(ctx, TNSK_ERR_INVALID, "stream: NULL argument");
    if (!is_m1(params->method))
        return fail(ctx, TNSK_ERR_UNSUPPORTED,
                    "stream: turnstile updates need stored sketches (TNSK_GENERAL or TNSK_CROSSCORR)");
    double* const outs[1] = {out};
    double* const pers[1] = {per_rep};
    tnsk_plan* p = nullptr;
    st = create_plan(ctx, 1, net, params, outs, per_rep ? pers : nullptr, true, &p);
    if (st != TNSK_OK) return st;
    p->no_graph = true;  // runs partial sequences: no graph of the whole plan
    st = launch_plan(ctx, p->plan, p->dev, p->fp64, nullptr);
    if (st != TNSK_OK) {
        tnsk_plan_destroy(p);
        return st;
    }
    tnsk_stream* s = new tnsk_stream();
    s->plan = p;
    *out_stream = s;
    return TNSK_OK;
}

tnsk_status tnsk_stream_update(tnsk_ctx* ctx, tnsk_stream* s, int64_t n, const int32_t* tensor, const int64_t* index,
                               const double* delta) {
    tnsk_status st = check_ctx(ctx);
    if (st != TNSK_OK) return st;
    if (!s) return fail(ctx, TNSK_ERR_INVALID, "stream: NULL");
    if (s->plan->device != ctx->device) return fail(ctx, TNSK_ERR_INVALID, "stream made on another device");
    if (n < 0 || (n > 0 && (!tensor || !index || !delta))) return fail(ctx, TNSK_ERR_INVALID, "stream: bad update list");
    if (n == 0) return TNSK_OK;
    const tnsk_plan* p = s->plan;
    ctx->prof.begin(TNSK_K_M1_SCATTER, ctx->stream);
    TNSK_CUDA(launch_m1_updates(p->plan, p->dev, n, tensor, index, delta, p->fp64, ctx->d_err, ctx->stream));
    ctx->prof.end(ctx->stream);
    return TNSK_OK;
}

tnsk_status tnsk_stream_estimate(tnsk_ctx* ctx, tnsk_stream* s) {
    tnsk_status st = check_ctx(ctx);
    if (st != TNSK_OK) return st;
    if (!s) return fail(ctx, TNSK_ERR_INVALID, "stream: NULL");
    const tnsk_plan* p = s->plan;
    if (p->device != ctx->device) return fail(ctx, TNSK_ERR_INVALID, "stream made on another device");
    const BatchPlan& plan = p->plan;
    unsigned char* base = p->dev;
    cudaStream_t cs = ctx->stream;
    // per-rep estimates start from zero (some transform paths accumulate into them);
    // the sketches, which follow them in the zeroed region, are kept
    TNSK_CUDA(cudaMemsetAsync(base + plan.yrep_off, 0, plan.m1.xs_off - plan.yrep_off, cs));
    Profiler& pf = ctx->prof;
    pf.begin(TNSK_K_M1_SPECTRUM, cs);
    TNSK_CUDA(launch_m1_spectra(plan, base, base + plan.m1.xs_off,
                                p->fp64 ? (const void* const*)ctx->d_tw64 : (const void* const*)ctx->d_tw32, p->fp64,
                                cs));
    pf.end(cs);
    pf.begin(TNSK_K_COMBINE, cs);
    TNSK_CUDA(launch_combine((const CombineItem*)(base + plan.comb_off), plan.n_comb,
                             (const double*)(base + plan.yrep_off), cs));
    pf.end(cs);
    return TNSK_OK;
}

tnsk_status tnsk_stream_sketches(tnsk_stream* s, void** x, int64_t* count) {
    if (!s || !x || !count) return TNSK_ERR_INVALID;
    const tnsk_plan* p = s->plan;
    *x = p->dev + p->plan.m1.xs_off;
    *count = p->plan.m1.xs_count;
    return TNSK_OK;
}

tnsk_status tnsk_stream_destroy(tnsk_stream* s) {
    if (!s) return TNSK_ERR_INVALID;
    tnsk_status st = tnsk_plan_destroy(s->plan);
    delete s;
    return st;
}

tnsk_status tnsk_combine(tnsk_ctx* ctx, int32_t R, int64_t O, const double* per_rep, int32_t groups, double* out) {
    tnsk_status st = check_ctx(ctx);
    if (st != TNSK_OK) return st;
    if (R < 1 || O < 0 || groups < 1 || groups > 64 || R % groups != 0)
        return fail(ctx, TNSK_ERR_INVALID, "combine: need R >= 1, O >= 0, groups in [1, 64] dividing R");
    if (O == 0) return TNSK_OK;
    if (!per_rep || !out) return fail(ctx, TNSK_ERR_INVALID, "combine: NULL buffer");
    std::vector<CombineItem> items((size_t)O);
    for (int64_t o = 0; o < O; ++o) items[(size_t)o] = CombineItem{0, O, o, R, groups, out, nullptr};
    const size_t bytes = items.size() * sizeof(CombineItem);
    st = ensure_scratch(ctx, bytes);
    if (st != TNSK_OK) return st;
    // pageable host staging: the copy has read `items` when it returns
    TNSK_CUDA(cudaMemcpyAsync(ctx->scratch, items.data(), bytes, cudaMemcpyHostToDevice, ctx->stream));
    ctx->prof.begin(TNSK_K_COMBINE, ctx->stream);
    TNSK_CUDA(launch_combine((const CombineItem*)ctx->scratch, (int)O, per_rep, ctx->stream));
    ctx->prof.end(ctx->stream);
    return TNSK_OK;
}

tnsk_status tnsk_probe_shared_atomics(tnsk_ctx* ctx, double* updates_per_s) {
    if (!updates_per_s) return TNSK_ERR_INVALID;
    tnsk_status st = check_ctx(ctx);
    if (st != TNSK_OK) return st;
    float* sink = nullptr;
    if (cudaMalloc((void**)&sink, sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, TNSK_ERR_OOM, "probe allocation failed");
    }
    cudaError_t e = run_probe_shared_atomics(sink, ctx->stream, updates_per_s);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "shared-atomic probe");
    return TNSK_OK;
}

tnsk_status tnsk_probe_shared_int_adds(tnsk_ctx* ctx, double* updates_per_s) {
    if (!updates_per_s) return TNSK_ERR_INVALID;
    tnsk_status st = check_ctx(ctx);
    if (st != TNSK_OK) return st;
    float* sink = nullptr;
    if (cudaMalloc((void**)&sink, sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, TNSK_ERR_OOM, "probe allocation failed");
    }
    cudaError_t e = run_probe_shared_int_adds(sink, ctx->stream, updates_per_s);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(sink);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "shared integer-add probe");
    return TNSK_OK;
}

tnsk_status tnsk_estimate(tnsk_ctx* ctx, const tnsk_network* net, const tnsk_params* params, double* out,
                          double* per_rep) {
    if (!ctx || !net || !params) return TNSK_ERR_INVALID;
    if (params->prec == TNSK_PREC_AUTO) return estimate_auto(ctx, net, params, out, per_rep);
    return run_batch(ctx, 1, net, params, &out, &per_rep, nullptr);
}

tnsk_status tnsk_auto_report(tnsk_ctx* ctx, int32_t* fp64_reps, double* max_rel_bound) {
    if (!ctx) return TNSK_ERR_INVALID;
    if (fp64_reps) *fp64_reps = ctx->auto_fp64_reps;
    if (max_rel_bound) *max_rel_bound = ctx->auto_max_bound;
    return TNSK_OK;
}

tnsk_status tnsk_estimate_batch(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, const tnsk_params* params,
                                double* const* outs, double* const* per_reps) {
    if (!ctx) return TNSK_ERR_INVALID;
    return run_batch(ctx, B, nets, params, outs, per_reps, nullptr);
}

tnsk_status tnsk_m1_sketch(tnsk_ctx* ctx, const tnsk_network* net, const tnsk_params* params, void* x) {
    if (!ctx || !net || !params) return TNSK_ERR_INVALID;
    if (!is_m1(params->method))
        return fail(ctx, TNSK_ERR_INVALID, "m1_sketch needs TNSK_GENERAL or TNSK_CROSSCORR");
    if (!x) return fail(ctx, TNSK_ERR_INVALID, "null sketch buffer");
    return run_batch(ctx, 1, net, params, nullptr, nullptr, x);
}

}  // extern "C"
