// plan.cuh -- host-side network validation and launch planning.
#pragma once

#include <string>
#include <vector>

#include "kernels.cuh"
#include "method2.cuh"

namespace tnsk {

// Methods that run on the method-1 kernels: method 1 and the cross-correlation
// estimator (the same sketches with another choice of complemented modes).
inline bool is_m1(int method) { return method == TNSK_GENERAL || method == TNSK_CROSSCORR; }

// A validated network (Def. "Tensor contraction", Def. "TNC"), 0-based modes.
struct NetInfo {
    int p = 0, q = 0, t = 0;
    std::vector<int> mode_off;      // [p+1]
    std::vector<int64_t> dims;      // [q]
    std::vector<int> tensor_of;     // [q]
    std::vector<int> edge_of;       // [q] edge or -1 (open)
    std::vector<int> side_of;       // [q] 0: first mode u (C), 1: second mode v (C')
    std::vector<int> open_pos;      // [q] position in the open list or -1
    std::vector<int64_t> numel;     // [p]
    std::vector<int64_t> open_tot;  // [p] O_k
    std::vector<int64_t> eoff;      // [t+1] edge table offsets
    int64_t L = 0;                  // sum of edge dims
    int64_t O = 1;                  // output entries
    int log2m = 0;
    bool idx32 = true;
    std::vector<const tnsk_rung*> rung;  // [p] grouped tensors (NULL: stored)
    std::vector<char> zero;              // [p] tensor given as all zeros (data NULL, streams only)
    std::vector<char> diag;              // [p] diagonal copy tensor of WLOG 1 (not stored)
    // method 2: rooted tree (children in mode order, footnote to Gamma(k))
    int root = -1;
    std::vector<int> parent, parent_mode, parent_edge, height;
    std::vector<std::vector<int>> child, child_mode, child_edge;
    int max_height = 0;
};

struct Arena {
    size_t used = 0;
    size_t take(size_t bytes, size_t align = 256);
};

struct M1Plan {
    int n_nets = 0;
    size_t tens_off = 0, nets_off = 0, work_off = 0, opens_off = 0, items_off = 0;
    size_t xs_off = 0, spec_off = 0, sexp_off = 0;
    int64_t xs_count = 0;  // sketch entries of all networks (FP32 or FP64)
    int n_work = 0, n_items = 0;
    // scatter work items by tensor order class (order <= 2, 4, 6, 12) and kernel: one
    // launch per list with its own unrolled width and shared-memory size. List
    // c + kOrderClasses * k: k = 0 the FP32 / FP64 atomic kernel (FP64 sketches, and
    // items whose bins go straight to global memory), k = 1 / 2 the fixed-point kernel
    // (FP32 sketches with privatised bins; 1: four entries per 16-byte load, 2: one),
    // k = 3 the fixed-point fiber kernel (whole fibers of a short contracted last mode)
    static constexpr int kOrderClasses = 4;
    static constexpr int kScatterLists = 4 * kOrderClasses;
    static_assert(kScatterLists == TNSK_SCATTER_LISTS, "tnsk_schedule covers every scatter list");
    int work_first[kScatterLists] = {};
    int work_count[kScatterLists] = {};
    size_t class_smem[kScatterLists] = {16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16, 16};
    int max_log2m = 0;
    // items of the warp-per-item spectrum kernel, by log2 m = 6 + slot, stored after
    // the n_items items of the block kernel
    static constexpr int kWarpSlots = 5;
    int warp_first[kWarpSlots] = {0, 0, 0, 0, 0};
    int warp_count[kWarpSlots] = {0, 0, 0, 0, 0};
    // large-m items (two-pass FFT, then the product over bin blocks) and their spectra
    size_t lfft_off = 0, lprod_off = 0, lspec_off = 0;
    int n_lfft = 0, n_lprod = 0;
    size_t lrows_smem = 16;  // shared memory of the pass-2 kernel (largest group of rows)
    // mid-m closed networks (m1_spectrum_mid.cu): the same two item lists, spectra in
    // the same scratch; shared memory sized by the largest m
    size_t mfft_off = 0, mprod_off = 0;
    int n_mfft = 0, n_mprod = 0;
    int mid_max_log2m = 0;
    // row-sorted sketches of large tensors (m1_rowsort.cu): per (tensor, rep) descriptors,
    // CTA items and the sorted-row scratch; shared memory of m floats
    size_t rs_off = 0, rs_items_off = 0, rs_scratch_off = 0;
    int n_rs = 0, n_rs_items = 0;
    int64_t rs_max_m = 0;
    int rs_max_rows = 0;  // largest item's row count
    // diagonal copy tensors (WLOG 1): one item each
    size_t diag_off = 0;
    int n_diag = 0;
    int64_t diag_most = 0;  // largest n * R
};

struct BatchPlan {
    Arena arena;
    std::vector<unsigned char> host_desc;
    size_t desc_off = 0;
    size_t zero_off = 0, zero_bytes = 0;
    size_t sketch_user_bytes = 0;
    size_t reqs_off = 0;
    int n_reqs = 0;
    int64_t n_table_rows = 0;  // (request, rep) rows
    size_t tabs_off = 0;
    size_t yrep_off = 0;
    int64_t yrep_n = 0;  // per-rep estimates at yrep_off; the magnitude sums follow them
    size_t comb_off = 0;
    int n_comb = 0;
    int m1_reps = 0;  // repetitions of the first method-1 network (turnstile streams)
    M1Plan m1;
    M2Plan m2;
};

// Launches the spectrum kernels of every method-1 item of the plan (rows a3 + a4).
// Launches the scatter of every method-1 work item (row a2), one launch per order class.
cudaError_t launch_m1_scatters(const BatchPlan& plan, unsigned char* base, void* xs, bool fp64, cudaStream_t s);
// The scatter launch of one list (class + kOrderClasses x kernel kind) alone.
cudaError_t launch_m1_scatter_list(const BatchPlan& plan, unsigned char* base, void* xs, bool fp64, int list,
                                   cudaStream_t s);
// Turnstile updates of a one-network method-1 plan's stored sketches (every rep).
cudaError_t launch_m1_updates(const BatchPlan& plan, unsigned char* base, int64_t n, const int32_t* tensor,
                              const int64_t* index, const double* delta, bool fp64, int* err, cudaStream_t s);
cudaError_t launch_m1_spectra(const BatchPlan& plan, unsigned char* base, const void* xs, const void* const* tws,
                              bool fp64, cudaStream_t s);
// Row-sorted sketches of the plan's large FP32 tensors added into xs (m1_rowsort.cu).
cudaError_t launch_m1_rowsort(const BatchPlan& plan, unsigned char* base, float* xs, cudaStream_t s);
// Sketches of the plan's diagonal copy tensors (WLOG 1) added into xs (every rep).
cudaError_t launch_m1_diag(const BatchPlan& plan, unsigned char* base, void* xs, bool fp64, cudaStream_t s);

// zero_ok: a tensor with data NULL is all zeros (turnstile streams fed by updates);
// diag (NULL or [p]): tensors that are diagonal copy tensors of WLOG 1 (data NULL)
tnsk_status validate(const tnsk_network& net, const tnsk_params& prm, NetInfo& info, std::string& why,
                     bool zero_ok = false, const char* diag = nullptr);
// True when the driver's tensor-map encoder is available (streaming tensor-core path).
bool tensor_maps_available();
// Encodes the plan's tensor maps into its host descriptor block once the device
// base address of the plan's scratch is fixed (before the descriptor upload).
tnsk_status finalize_plan(BatchPlan& plan, unsigned char* base, std::string& err);
// Hands an uploaded plan's staged descriptor block back for the calling thread's next
// plan (its memory is reused instead of allocated and faulted in again); H is left empty.
void recycle_host_desc(std::vector<unsigned char>& H);
// sched: the scatter schedule (tnsk.h), NULL = the default one. rep_stride: per
// network, the row stride of its per-rep output for method 2 (NULL or 0: 1; an output
// entry of a network with open legs estimated as its own full network, see api.cu).
tnsk_status plan_batch(const std::vector<NetInfo>& infos, const tnsk_network* nets, const tnsk_params* params,
                       double* const* outs, double* const* per_reps, bool fp64, bool sketch_only, BatchPlan& plan,
                       std::string& err, const tnsk_schedule* sched = nullptr,
                       const int64_t* rep_stride = nullptr);

}  // namespace tnsk
