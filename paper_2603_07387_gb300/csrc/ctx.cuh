// ctx.cuh -- the library context (tnsk_ctx) and the host helpers every C-ABI
// source uses: error recording, context checks, the shared scratch arena.
#pragma once

#include <string>

#include "kernels.cuh"

struct tnsk_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string last_error;
    tnsk_status deferred = TNSK_OK;
    // scratch arena, grown on demand, reused by every call (stream ordered)
    unsigned char* scratch = nullptr;
    size_t scratch_bytes = 0;
    // tensors rewritten for the acyclic method (WLOG 2 / 3), grown on demand, stream ordered
    unsigned char* norm = nullptr;
    size_t norm_bytes = 0;
    // twiddles tw[k] = exp(-2 pi i k/m), k < m/2, for m = 2^l, l = 0..16
    void* tw32[17] = {};
    void* tw64[17] = {};
    const void** d_tw32 = nullptr;  // device arrays of the pointers above
    const void** d_tw64 = nullptr;
    int* d_err = nullptr;  // device error word
    // second stream for method 1 while method 2 runs on the ctx stream, and the
    // events that fork it from and join it back into the ctx stream
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    tnsk::Profiler prof;
    // fault injection for tests (tnsk_debug_inject): consumed by the next launch sequence
    int inject = 0;
    // the last TNSK_PREC_AUTO estimate: reps taken in FP64, largest relative bound
    int32_t auto_fp64_reps = 0;
    double auto_max_bound = 0.0;
    // per-rep buffer of TNSK_PREC_AUTO calls made without one (grown on demand)
    double* aux = nullptr;
    size_t aux_bytes = 0;
    // the predictor's small device buffers (features, inputs and outputs, pilot
    // estimates), grown on demand and reused, so a parameter choice allocates nothing
    unsigned char* work = nullptr;
    size_t work_bytes = 0;
    // method 2 with open legs: the tensors with open modes rewritten open modes first
    // (their slices contiguous), then the job descriptors; grown on demand, stream ordered
    unsigned char* open_buf = nullptr;
    size_t open_bytes = 0;
};

namespace tnsk {
// records msg as the ctx's last error and returns st
tnsk_status ctx_fail(tnsk_ctx* ctx, tnsk_status st, const std::string& msg);
tnsk_status ctx_cuda_fail(tnsk_ctx* ctx, cudaError_t e, const char* where);
// non-null, no deferred device error, its device current
tnsk_status ctx_check(tnsk_ctx* ctx);
// the ctx scratch arena holds at least `bytes` (stream-ordered reuse)
tnsk_status ctx_ensure_scratch(tnsk_ctx* ctx, size_t bytes);
// the ctx work buffer (ctx->work) holds at least `bytes` (stream-ordered reuse)
tnsk_status ctx_ensure_work(tnsk_ctx* ctx, size_t bytes);
}  // namespace tnsk
