// normalize.cuh -- the WLOG rewrites of Sec. 4.1 done by the library.
//
// WLOG 1 (TNSK_GENERAL, TNSK_CROSSCORR): the modes that contractions force equal
// fall into classes; a class of three or more modes (some mode in two or more
// contractions) becomes a diagonal copy tensor delta(i, ..., i) of order d joined to
// each member g_1 < ... < g_d. Copy tensors are appended after the p tensors (classes
// by lowest mode id); the contractions are those of the two-mode classes in their
// order (a repeated pair once), then (g_j, c_j) per copy tensor. Copy tensors are not
// stored: their n nonzeros are sketched directly (m1_diag_kernel).
//
// Method 2 (Sec. 4.4) needs every contraction to join two different tensors and
// at most one contraction between any two tensors. A TNSK_ACYCLIC network that
// breaks either is rewritten before planning:
//   WLOG 2: a contraction inside tensor X_k is summed exactly over its diagonal and
//           both modes leave X_k;
//   WLOG 3: the r >= 2 contractions e_1 < ... < e_r (edge-list order) between two
//           tensors become one: in each tensor their modes are replaced by one mode
//           at the place of the lowest of them, of size prod n_{e_j}, index
//           row-major over (i_{e_1}, ..., i_{e_r}); the merged contraction stands
//           where e_1 stood, with e_1's first endpoint first.
// Tensors keep their order and count; other modes and contractions keep their
// relative order. A tensor whose modes only need a reshape (merged modes already
// adjacent and in edge order, no trace) keeps its data; the others are written
// once by normalize_kernel into a buffer the caller provides (FP64 sources stay
// FP64, FP32 and BF16 sources become FP32; diagonal sums accumulate in FP64).
#pragma once

#include <string>
#include <vector>

#include "common.cuh"

namespace tnsk {

struct NormJob {
    const void* src;
    void* dst;
    int64_t numel;                      // output entries
    int64_t dim[TNSK_MAX_ORDER];        // output modes before the merge reshape, row-major
    int64_t str[TNSK_MAX_ORDER];        // their strides in the source (elements)
    int64_t ddim[TNSK_MAX_ORDER / 2];   // traced pairs: dim, and the sum of the pair's strides
    int64_t dstr[TNSK_MAX_ORDER / 2];
    int32_t n, nd, src_dtype, dst_f64;
};

struct NormNet {
    tnsk_network net{};  // the rewritten network (points into the vectors below)
    std::vector<tnsk_tensor> X;
    std::vector<std::vector<int64_t>> dims;
    std::vector<int32_t> edges;
    std::vector<int> job;  // per tensor: index into NormBatch::jobs, or -1
};

struct NormBatch {
    bool used = false;                // some network was rewritten
    std::vector<NormNet> nets;        // per batch network (empty net.X: not rewritten)
    std::vector<tnsk_network> view;   // the networks to plan: rewritten or the caller's
    std::vector<std::vector<char>> diag;  // per network: [p'] 1 = WLOG 1 copy tensor (empty: none)
    std::vector<NormJob> jobs;        // host descriptors (dst set by normalize_bind)
    std::vector<size_t> dst_off;      // per job: its output's offset in the buffer
    size_t desc_off = 0;              // descriptors after the outputs
    size_t bytes = 0;                 // buffer size
    int64_t most = 0;                 // largest job output
};

// Host: rewrites the TNSK_ACYCLIC networks that need WLOG 2 / 3 and the method-1
// networks (TNSK_GENERAL, TNSK_CROSSCORR) that need WLOG 1. Networks that fail the
// basic checks of tnsk_estimate are left as they are (planning reports them).
// TNSK_ERR_UNSUPPORTED when a grouped (rung) tensor would have to be rewritten or a
// copy tensor would have more than TNSK_MAX_ORDER modes.
tnsk_status normalize_batch(int B, const tnsk_network* nets, const tnsk_params* params, NormBatch& nb,
                            std::string& why);
// Points the rewritten tensors and the jobs' outputs into base (>= nb.bytes, 256-byte aligned).
void normalize_bind(NormBatch& nb, unsigned char* base);
// One launch for all jobs (descriptors at d_jobs, device).
cudaError_t launch_normalize(const NormJob* d_jobs, int n, int64_t most, cudaStream_t s);

}  // namespace tnsk
