// kernels.cuh -- launchers of the libtnsk kernels (host-callable).
#pragma once

#include <vector>

#include "common.cuh"

namespace tnsk {

// Optional per-launch CUDA-event timing (tnsk_profile). begin/end bracket one
// launch on the stream; events come from a reusable pool.
struct Profiler {
    bool on = false;
    struct Rec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void begin(int kind, cudaStream_t s) {
        if (!on) return;
        Rec r{kind, get(), get()};
        cudaEventRecord(r.a, s);
        recs.push_back(r);
    }
    void end(cudaStream_t s) {
        if (!on || recs.empty()) return;
        cudaEventRecord(recs.back().b, s);
    }
    ~Profiler() {
        for (auto& r : recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

struct CombineItem {  // one output entry of one network
    int64_t y_off;    // per-rep estimates [R][O]
    int64_t O;
    int64_t o;
    int32_t R;
    int32_t groups;
    double* out;
    double* per_rep;  // optional [R][O]: rep r's value of entry o at r * ps + o
    int64_t ps;       // per_rep row stride (O, or the caller's for an expanded network)
};

// One table row per (request, rep); rows = sum of the requests' R (crow prefix).
cudaError_t launch_draw_tables(const TabReq* d_reqs, int nreq, int64_t rows, uint32_t* d_out, cudaStream_t s);
cudaError_t launch_count_sketch(uint64_t seed, uint64_t rep, uint64_t tid, int64_t n, int64_t m, int32_t* bins,
                                int8_t* signs, cudaStream_t s);
cudaError_t launch_m1_scatter(const M1Tensor* d_tens, const M1Net* d_nets, const M1Work* d_work, int n_work,
                              const uint32_t* d_tabs, void* d_xs, bool fp64, size_t smem, int max_order,
                              cudaStream_t s);
// FP32 sketches, privatised bins in fixed point (m1_scatter_fx.cu); vec4: every item's
// tensor is FP32, 16-byte aligned, last dim a multiple of 4
cudaError_t launch_m1_scatter_fx(const M1Tensor* d_tens, const M1Net* d_nets, const M1Work* d_work, int n_work,
                                 const uint32_t* d_tabs, float* d_xs, size_t smem, int max_order, bool vec4,
                                 cudaStream_t s);
// CTA slots of the row-sorted sketch kernel on the current device (SMs x CTAs per SM)
int64_t m1_rowsort_slots();
// entries per CTA batch of the fixed-point kernel for tensors of order <= max_order
int m1_fx_batch(int max_order, bool vec4 = true);
// the fiber kernel (FP32 sketches, a contracted last mode of L <= 16 indices): whole
// fibers per thread, entries per CTA batch
cudaError_t launch_m1_scatter_fiber(const M1Tensor* d_tens, const M1Net* d_nets, const M1Work* d_work, int n_work,
                                    const uint32_t* d_tabs, float* d_xs, size_t smem, int max_order,
                                    cudaStream_t s);
int64_t m1_fiber_batch(int L);
cudaError_t launch_m1_spectrum(const M1Tensor* d_tens, const M1Net* d_nets, const OpenMode* d_opens,
                               const int2* d_items, int n_items, const void* d_xs, const void* const* d_tws,
                               void* d_spec, int* d_sexp, double* d_yrep, bool fp64, int max_log2m,
                               cudaStream_t s);
// m above one CTA's shared memory, no open legs: pass 1 of the packed four-step FFT
// per (net, rep, sketch) into d_lspec, then pass 2 with the product and bin sum per
// (net, rep, pair of rows)
cudaError_t launch_m1_large(const M1Tensor* d_tens, const M1Net* d_nets, const int4* d_fft_items, int n_fft,
                            const int4* d_prod_items, int n_prod, size_t rows_smem, const void* d_xs,
                            const void* const* d_tws, void* d_lspec, double* d_yrep, bool fp64, cudaStream_t s);
// the large path's pass 2: shared memory for G sketches' pairs of rows, and the G
// that fits (at most p)
size_t m1_large_rows_smem(int log2m, int G, bool fp64);
int m1_large_rows_group(int log2m, int p, bool fp64);
// closed networks at 2^11 <= m <= 2^14: one CTA per (net, rep, sketch) transform into
// the half spectra in d_lspec, then the product and bin sum per (net, rep, bin block)
cudaError_t launch_m1_mid(const M1Tensor* d_tens, const M1Net* d_nets, const int4* d_fft_items, int n_fft,
                          const int4* d_prod_items, int n_prod, int max_log2m, const void* d_xs,
                          const void* const* d_tws, void* d_lspec, double* d_yrep, bool fp64, cudaStream_t s);
// FP32 networks, 2^6 <= m = 2^log2m <= 2^10: one warp per item (open legs: spectra
// stored to d_spec / d_sexp in the block kernel's layout)
cudaError_t launch_m1_spectrum_warp(const M1Tensor* d_tens, const M1Net* d_nets, const OpenMode* d_opens,
                                    const int2* d_items, int n_items, const void* d_xs, const void* const* d_tws,
                                    void* d_spec, int* d_sexp, double* d_yrep, int log2m, cudaStream_t s);
cudaError_t launch_combine(const CombineItem* d_items, int n_items, const double* d_yrep, cudaStream_t s);
// measurement aid: random-bin FP32 shared-memory atomic adds per second (waits for s)
cudaError_t run_probe_shared_atomics(float* sink, cudaStream_t s, double* updates_per_s);
// measurement aid: random-bin 32-bit integer shared-memory adds per second (waits for s)
cudaError_t run_probe_shared_int_adds(float* sink, cudaStream_t s, double* updates_per_s);

}  // namespace tnsk
