/*
 * tnsk.h -- C ABI of libtnsk: GB300 (sm_103a) sketching estimators for tensor
 * network contraction, after "Approximating Tensor Network Contraction with
 * Sketches" (Heddes, Nunes, Givargis, Nicolau; arXiv 2603.07387).
 *
 * Problem (Sec. 1, Def. "Tensor contraction", Def. "Tensor product", Def. "TNC"):
 * tensors X_1..X_p, a set E of mode pairs (u, v) with u != v and n_u = n_v, modes
 * numbered globally across X_1 x ... x X_p in order (0-based here, 1-based in the
 * paper). tc(X, E)(i_K') = sum_{i_K} X(i) prod_{(u,v) in E} [i_u = i_v], where K'
 * are the open (uncontracted) modes. The library returns a randomised estimate
 * (Def. "ATNC": error relative to ||X||_F = prod_k ||X_k||_F):
 *   TNSK_GENERAL  method 1, any network incl. cyclic ones (Sec. 4.2, Eq. 1, Alg. 1),
 *                 complement count sketches, FFT-domain composition;
 *   TNSK_ACYCLIC  method 2, acyclic full networks (Sec. 4.4, Eq. 2, Alg. 2, 4, 5),
 *                 recursive sketches evaluated leaves to root.
 * Repetitions are combined by the median of group means (Theorem 1, median trick);
 * open output entries follow Corollary "full-to-partial-tc".
 *
 * Conventions for every call:
 *  - Tensor data, outputs and per-rep buffers are DEVICE pointers on the ctx's
 *    device; sizes and descriptors are host memory read during the call only.
 *  - Tensors are row-major (the paper's vec(): last mode fastest, Sec. 2).
 *  - Calls enqueue work on the ctx stream and return before it completes. The
 *    caller keeps inputs alive and outputs untouched until the stream reaches
 *    the work (e.g. tnsk_sync). Errors the host can see are returned at once;
 *    device-side errors (exhausted waits, failed bounds checks) are recorded in
 *    the ctx and returned by tnsk_sync or the next call.
 *  - The caller owns every buffer it passes. The library allocates only its own
 *    scratch (cached in the ctx, freed by tnsk_destroy) and keeps no caller
 *    pointer after the work that uses it completes.
 *  - One ctx per host thread; a ctx is not thread safe.
 *  - Limits: m a power of two, 1 <= m <= 65536; tensor order <= 12; reps <= 65536.
 * Hash contract (the paper fixes only 2-wise bins and 4-wise signs, Sec. 2.1):
 * SplitMix64-keyed Carter-Wegman polynomials over P = 2^61 - 1, specified in
 * the comment of tnsk_count_sketch below.
 */
#ifndef TNSK_H
#define TNSK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TNSK_OK = 0,
    TNSK_ERR_INVALID = -1,      /* malformed network or parameters */
    TNSK_ERR_CYCLIC = -2,       /* TNSK_ACYCLIC on a network with a cycle */
    TNSK_ERR_UNSUPPORTED = -3,  /* valid, but outside the library's limits */
    TNSK_ERR_CUDA = -4,         /* a CUDA runtime call failed */
    TNSK_ERR_OOM = -5,          /* scratch allocation failed */
    TNSK_ERR_TIMEOUT = -6,      /* a device-side bounded wait gave up */
    TNSK_ERR_UNREACHABLE = -7   /* no parameters meet the requested error */
} tnsk_status;

typedef enum { TNSK_F64 = 0, TNSK_F32 = 1, TNSK_BF16 = 2 } tnsk_dtype;
/* TNSK_CROSSCORR: the earlier estimator Sec. 4.2 contrasts with method 1 (its two
 * examples), kept for comparison: every contraction gets one plain count sketch,
 * every tensor its tensor sketch, and the sketches are combined by the circular
 * cross-correlation x_1 * x_2 * ... * x_p taken left to right, whose first
 * component is the estimate. In the Fourier domain the chain conjugates tensor k's
 * spectrum when p - 1 - k is odd, which the library computes as method 1 with the
 * complement count sketch on every contracted mode of those tensors (and the plain
 * one on all others), edge tables as method 1's. Unbiased when every contraction
 * joins a conjugated and an unconjugated tensor (e.g. a chain); otherwise biased
 * (on the triangle tr(XYZ) the expectation is about 2 tc / m). Same limits, layout
 * and calls as TNSK_GENERAL (tnsk_estimate, batches, plans, tnsk_m1_sketch,
 * streams); tnsk_choose_params and tnsk_estimate_static refuse it. */
typedef enum { TNSK_GENERAL = 1, TNSK_ACYCLIC = 2, TNSK_CROSSCORR = 3 } tnsk_method;
/* Arithmetic of the sketches and transforms (the paper fixes none).
 * FP32: sketches accumulated exactly in integers per batch of entries and rounded to
 *   FP32 (method 1: every entry quantised to 2^-30 of its batch's sum |x|), FFTs and
 *   products in FP32 (per-tensor power-of-two scaling), method 2's sketched product
 *   mat(X_k) V on the tensor cores with a 3-pass TF32 split (FP32 accuracy),
 *   per-rep estimates and combination in FP64.
 * BF16: tensors stored as TNSK_BF16 (a stored tensor of another dtype returns
 *   TNSK_ERR_UNSUPPORTED; grouped tensors are FP32 and unsupported), read as they
 *   are; method 2's sketched product on BF16 tensor cores (tcgen05 kind::f16) with
 *   X as stored and V as the sum of three BF16 parts, FP32 accumulation, so the
 *   result is that of FP32 arithmetic on the BF16 values; everything else as FP32.
 * FP64: everything in FP64 (for high-dynamic-range sketches). */
/* AUTO (tnsk_estimate only; method 1, no open legs): the FP32 path, then the FP64 path
 *   for the reps whose FP32 transforms may be inexact. Every spectral kernel also
 *   returns the rep's magnitude sum A_r = (1/m) sum_j (|Re| + |Im|)(prod_k F x_k(j))
 *   (at most sqrt 2 times the sum of the moduli); the FP32
 *   rounding of the transforms and of the products is at most about
 *   c32 A_r, c32 = (p + 2 log2 m + 8) 2^-24 (p as given), so a rep with c32 A_r > 2^-17 |y_r| (a
 *   sketch whose spectrum has a high dynamic range and cancels in the sum) is flagged.
 *   The smallest range of reps holding every flagged rep is recomputed by the FP64
 *   path (same hash functions: FP64 sketches from the same inputs, FP64 transforms),
 *   and the estimate is the combination of the resulting per-rep values.
 *   tnsk_auto_report gives the number of reps taken in FP64 and the largest remaining
 *   relative bound, c A_r / |y_r| over the reps (c = c32 or its FP64 counterpart). */
typedef enum { TNSK_PREC_FP32 = 0, TNSK_PREC_BF16 = 1, TNSK_PREC_FP64 = 2, TNSK_PREC_AUTO = 3 } tnsk_precision;

typedef struct tnsk_ctx tnsk_ctx;

/* A grouped tensor (Sec. 4.1, grouping: two tensors contracted exactly along their
 * shared mode become one tensor): R((i, j), (k, l)) = sum_s A(i, s, k) B(j, s, l),
 * an order-2 tensor of dims [a*b, c*d] (first index i*b + j, second k*d + l). The
 * rung of two tensor trains joined on their physical legs has this form. Entries are
 * never stored: the method-2 sketch product computes them from A and B (FP32 sums in
 * the order s = 0, 1, ...: the values contract_pairs would write). */
typedef struct {
    const void* A;          /* device FP32 [a][s][c], row-major */
    const void* B;          /* device FP32 [b][s][d], row-major */
    int64_t a, s, c, b, d;  /* all >= 1 */
} tnsk_rung;

typedef struct {
    int32_t order;          /* q_k >= 0 (0 = scalar) */
    const int64_t* dims;    /* [order] host */
    const void* data;       /* device, row-major, numel = prod dims; NULL with rung */
    tnsk_dtype dtype;
    const tnsk_rung* rung;  /* host; NULL for a tensor stored at data. Else the tensor
                               is the grouped tensor above: order 2, dims
                               [a*b, c*d], dtype TNSK_F32, data NULL; accepted by
                               TNSK_ACYCLIC in FP32 where it is an inner node of the
                               rooted tree (neither a leaf nor the root) and the
                               column pair's fast index (d, or b when the parent mode
                               is the second) is a multiple of 32, the staged B factor
                               within 64 KiB and s <= 16; elsewhere TNSK_ERR_UNSUPPORTED */
} tnsk_tensor;

typedef struct {
    int32_t p;              /* number of tensors, >= 1 */
    const tnsk_tensor* X;   /* [p] host */
    int32_t t;              /* |E| */
    const int32_t* edges;   /* [2t] host: pairs (u, v) of global mode ids; the
                               first mode u gets the count sketch C, v its
                               complement C' (Sec. 4.2) */
    int32_t n_open;         /* |K'| */
    const int32_t* open;    /* [n_open] host: permutation of K' giving the output
                               mode order; output is row-major over it */
} tnsk_network;

typedef struct {
    int64_t m;              /* sketch size */
    int32_t reps;           /* independent repetitions R */
    int32_t groups;         /* median of `groups` group means; 1 = plain mean */
    uint64_t seed;          /* hash seed */
    tnsk_method method;
    int32_t root;           /* method 2 root tensor; -1 = the tensor with the
                               fewest entries (lowest index on ties) */
    tnsk_precision prec;
    int32_t rep0;           /* index of the first repetition: the call draws the hash
                               functions of reps rep0 .. rep0 + reps - 1, so shards of
                               one estimate (e.g. on several GPUs) can be combined;
                               0 for a whole estimate */
} tnsk_params;

/* Create a context on `device` whose work goes to `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream). */
tnsk_status tnsk_create(tnsk_ctx** ctx, int device, void* cuda_stream);
/* Wait for the ctx's work, free its scratch and the ctx. */
tnsk_status tnsk_destroy(tnsk_ctx* ctx);
/* Rebind the ctx to another stream of the same device. */
tnsk_status tnsk_set_stream(tnsk_ctx* ctx, void* cuda_stream);

/* Count sketch table of the hash contract (Sec. 2.1, Def. "Count sketch") for
 * repetition `rep` and table id `tid`:
 *   sm(x)    SplitMix64 output for state x; K = sm(sm(sm(seed) ^ rep) ^ tid);
 *   c(r,j) = sm(K ^ (8r + j)) folded into [0, P), P = 2^61 - 1;
 *   bins[i]  = ((c(0,1) i + c(0,0)) mod P) mod m                  (2-wise)
 *   signs[i] = +1 if (c(1,3) i^3 + c(1,2) i^2 + c(1,1) i + c(1,0)) mod P is even,
 *              -1 otherwise                                       (4-wise)
 * Table ids: method 1 edge e: (1<<56)|e; method 2 edge e: (2<<56)|e; method 2
 * padding slot j of tensor k: (3<<56)|(k<<24)|j; method 2 tensor sketch T_{2^l,j}
 * side s of tensor k: (4<<56)|(k<<24)|(l<<16)|(j<<1)|s.
 * bins: device int32[n]; signs: device int8[n]. */
tnsk_status tnsk_count_sketch(tnsk_ctx* ctx, uint64_t seed, uint64_t rep, uint64_t tid, int64_t n,
                              int64_t m, int32_t* bins, int8_t* signs);

/* Method-1 sketches x_k = T_k vec(X_k) of every tensor (Eq. 1; Alg. 1 "x_k <- T_k
 * vec(X_k)"; hash form of Alg. 3) for reps 0..R-1 of params. Output x: device,
 * float (FP32) or double (FP64) by params->prec, laid out [R][sum_k O_k m] with
 * tensor k's block [O_k][m] (O_k = product of its open dims, row-major in the
 * tensor's mode order), blocks in tensor order. */
tnsk_status tnsk_m1_sketch(tnsk_ctx* ctx, const tnsk_network* net, const tnsk_params* params, void* x);

/* Estimate tc(X, E): out = device double[prod of open dims] (1 entry if full);
 * per_rep = device double[R][prod open dims] or NULL.
 * TNSK_GENERAL and TNSK_CROSSCORR networks may have hyperedges (a mode in two or
 * more contractions); the library applies WLOG 1 of Sec. 4.1 (the same in batches,
 * plans, streams and tnsk_m1_sketch): the modes that contractions force equal form
 * classes, and a class of three or more modes g_1 < ... < g_d becomes a diagonal
 * copy tensor delta(i, ..., i) of order d (dims n) joined to each g_j. The network
 * planned is: the caller's tensors, then one copy tensor per such class (classes by
 * lowest mode id); contractions: those of the two-mode classes in the caller's order
 * (a repeated pair kept once), then (g_j, c_j), j = 1..d, per copy tensor (c_j its
 * j-th mode). Hash tables follow that contraction list; the copy tensors are never
 * stored (their n nonzeros are sketched directly) and tnsk_m1_sketch writes their
 * sketches after the caller's tensors. At most TNSK_MAX_ORDER modes per class
 * (TNSK_ERR_UNSUPPORTED beyond); TNSK_ACYCLIC refuses hyperedges
 * (TNSK_ERR_UNSUPPORTED).
 * TNSK_ACYCLIC networks are first brought into the form Sec. 4.1 assumes (the
 * same in tnsk_estimate_batch and tnsk_plan_create):
 *   WLOG 2: a contraction whose two modes belong to one tensor is summed exactly
 *           over its diagonal and both modes leave that tensor;
 *   WLOG 3: the r >= 2 contractions e_1 < ... < e_r (order of `edges`) between
 *           one pair of tensors become one contraction: in each of the two
 *           tensors their modes are replaced by a single mode at the place of
 *           the lowest of them, of size prod_j n_{e_j}, index row-major over
 *           (i_{e_1}, ..., i_{e_r}) (the paper's example: vec(A) . vec(B)).
 * Tensors keep their order and count, other modes and contractions their relative
 * order; the merged contraction stands where e_1 stood, e_1's first endpoint
 * first. Method 2's hash functions and `root` refer to this rewritten network. A
 * tensor that needs more than a reshape is written once (FP64 stays FP64, FP32
 * and BF16 become FP32; diagonal sums in FP64) into a ctx-owned buffer (a
 * plan's own buffer for tnsk_plan_create), by a kernel the call enqueues before
 * the method's kernels. A cycle through three or more tensors still returns
 * TNSK_ERR_CYCLIC; a grouped (rung) tensor that would need the rewrite, or a
 * merged mode above 2^31 - 1, TNSK_ERR_UNSUPPORTED.
 * TNSK_ACYCLIC networks with open legs (tnsk_estimate and tnsk_estimate_batch; plans
 * refuse them): each output entry o, row-major over `open`, is the full estimate of
 * the network whose tensors are sliced at o's open indices (Corollary
 * "full-to-partial-tc"), all entries with the same hash functions. Every tensor with
 * open modes is first written once, open modes first, into a ctx-owned buffer (FP64
 * stays FP64, FP32 and BF16 become FP32); the entries then run in one batch, the
 * slices being the networks planned (WLOG 2 / 3 apply to them, `root` refers to their
 * tensors, the default root taking the smallest slice). per_rep, if given, receives
 * [R][O] as for method 1. At most 2^16 output entries per call (TNSK_ERR_UNSUPPORTED
 * beyond, and for an empty output or a grouped tensor with open modes). */
tnsk_status tnsk_estimate(tnsk_ctx* ctx, const tnsk_network* net, const tnsk_params* params, double* out,
                          double* per_rep);

/* The network tnsk_estimate plans for `net` under `params` after the WLOG rewrites
 * above, computed on the host only (no ctx, no device work): *p_out tensors, tensor
 * k of order order_out[k] with its dims next in dims_out (concatenated in tensor
 * order), copy_out[k] = 1 for a WLOG 1 copy tensor; *t_out contractions as pairs in
 * edges_out. Capacities: cap_tensors entries of order_out and copy_out, cap_dims of
 * dims_out, cap_edges pairs of edges_out. A network that needs no rewrite (or fails
 * the basic checks, which tnsk_estimate then reports) is returned as given.
 * Errors: TNSK_ERR_INVALID for NULL pointers or a capacity too small; the rewrite's
 * own TNSK_ERR_UNSUPPORTED cases as in tnsk_estimate. */
tnsk_status tnsk_rewrite(const tnsk_network* net, const tnsk_params* params, int32_t cap_tensors, int32_t* p_out,
                         int32_t* order_out, int32_t* copy_out, int64_t cap_dims, int64_t* dims_out, int32_t cap_edges,
                         int32_t* t_out, int32_t* edges_out);

/* B networks in one batch (one launch sequence for all). params[b], outs[b],
 * per_reps[b] (may be NULL, or hold NULL entries) as in tnsk_estimate. */
tnsk_status tnsk_estimate_batch(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, const tnsk_params* params,
                                double* const* outs, double* const* per_reps);

/* Row a9 on its own (Theorem 1's median trick): out[o] = the median of `groups`
 * contiguous group means of per_rep[r][o] over r < R (groups = 1: the mean; an
 * even count takes the mean of the two middle values), all in FP64. per_rep:
 * device double[R][O] (e.g. per-rep estimates gathered from several GPUs that
 * each ran a block of reps via tnsk_params.rep0); out: device double[O].
 * Errors: TNSK_ERR_INVALID when R < 1, O < 0, groups outside [1, 64] or not
 * dividing R, or a pointer is NULL while O > 0. */
tnsk_status tnsk_combine(tnsk_ctx* ctx, int32_t R, int64_t O, const double* per_rep, int32_t groups, double* out);

/* Turnstile streams (Sec. 4.2: method 1 stores the sketches x_k, so the general
 * turnstile model is served by applying each update X_k(i) += delta to every rep's
 * sketch of X_k, in O(q_k)). tnsk_stream_create sketches the network's tensors as
 * they are now (one method-1 network, params->method == TNSK_GENERAL, else
 * TNSK_ERR_UNSUPPORTED), writes the estimate to `out` (device, prod of open dims) and
 * `per_rep` (device [reps][O] or NULL), and keeps the sketches in memory owned by
 * the stream; once that work has run, the tensors are not read again. A tensor
 * whose data is NULL starts as all zeros: the sparse (COO) input path, where the
 * nonzeros arrive as updates, each costing O(q_k) per rep instead of a dense pass.
 * tnsk_stream_update applies n updates: tensor[u] (0-based tensor of the network),
 * index[u] (row-major flat entry index), delta[u]; all three device arrays [n],
 * read by the launch. An update out of range changes nothing and makes the next
 * tnsk_sync return TNSK_ERR_INVALID. Updates commute (atomic adds; FP32 sketches
 * add in an order that varies between runs). tnsk_stream_estimate recomputes `out`
 * and `per_rep` from the current sketches (transform, product, combination). All
 * three enqueue on the ctx stream. tnsk_stream_destroy waits for the device and
 * frees the stream. */
typedef struct tnsk_stream tnsk_stream;
tnsk_status tnsk_stream_create(tnsk_ctx* ctx, const tnsk_network* net, const tnsk_params* params, double* out,
                               double* per_rep, tnsk_stream** stream);
tnsk_status tnsk_stream_update(tnsk_ctx* ctx, tnsk_stream* stream, int64_t n, const int32_t* tensor,
                               const int64_t* index, const double* delta);
tnsk_status tnsk_stream_estimate(tnsk_ctx* ctx, tnsk_stream* stream);
/* The stream's stored sketches (sketches are linear in the tensors, Sec. 4.2): *x =
 * device pointer (owned by the stream) to *count FP32 or FP64 entries (params->prec),
 * laid out as tnsk_m1_sketch's output ([reps][sum_k O_k m], copy tensors of WLOG 1
 * after the caller's tensors; the count may include up to 3 entries of padding).
 * Several processes that each stream a part of the same tensors' entries, with the
 * same network and params, can sum these buffers (e.g. an all-reduce) and then call
 * tnsk_stream_estimate to estimate the whole: the sketch of a sum is the sum of the
 * sketches. Order the reduction after the stream's work on the ctx stream.
 * TNSK_ERR_INVALID for NULL arguments. */
tnsk_status tnsk_stream_sketches(tnsk_stream* stream, void** x, int64_t* count);
tnsk_status tnsk_stream_destroy(tnsk_stream* stream);

/* Per-kernel timing. While enabled, every kernel launch of the ctx is bracketed
 * by CUDA events recorded on the ctx stream. tnsk_profile_read waits for the
 * stream, writes the summed device time (ms) and the launch count of each kernel
 * kind (arrays of TNSK_KERNEL_KINDS entries, indexed by tnsk_kernel_kind) and
 * clears the records. Timing adds no synchronisation to the launch sequence. */
typedef enum {
    TNSK_K_TABLES = 0,      /* hash tables of all reps (a1) */
    TNSK_K_M1_SCATTER = 1,  /* method 1 signed scatter-add (a2), copy tensors included */
    TNSK_K_M1_SPECTRUM = 2, /* method 1 FFT, Hadamard product, bin sum (a3, a4) */
    TNSK_K_M2_LEAF = 3,     /* method 2 leaf count sketches (a5) */
    TNSK_K_M2_COMPOSE = 4,  /* method 2 Q_k composition (a6) */
    TNSK_K_M2_VBUILD = 5,   /* method 2 recursive-sketch columns (a7) */
    TNSK_K_M2_GEMM = 6,     /* method 2 sketched matrix-vector products (a7) */
    TNSK_K_M2_ROOT = 7,     /* method 2 root inner products (a8) */
    TNSK_K_COMBINE = 8,     /* median of group means (a9) */
    TNSK_K_M2_SCATTER = 9,  /* method 2 count-sketch scatter of the product rows (a7) */
    TNSK_K_PAIRS = 10,      /* exact pair contractions (tnsk_pairs_run) */
    TNSK_K_NORMALIZE = 11,  /* WLOG 2 / 3 rewrite of acyclic networks (Sec. 4.1) */
    TNSK_K_M2_PREP = 12,    /* method 2: TF32 parts of grouped tensors' factors, once per run (a7) */
    TNSK_KERNEL_KINDS = 13
} tnsk_kernel_kind;
tnsk_status tnsk_profile(tnsk_ctx* ctx, int32_t enable);
tnsk_status tnsk_profile_read(tnsk_ctx* ctx, double* ms, int64_t* launches);

/* A batch planned once and run many times. tnsk_plan_create validates the B
 * networks and lays out and uploads every launch descriptor into device memory
 * owned by the plan (cudaMalloc); each tnsk_plan_run enqueues the whole launch
 * sequence of tnsk_estimate_batch on the ctx stream, reading the tensors and
 * writing outs / per_reps at the addresses given at creation (new data in the
 * same buffers is picked up by the next run). The plan keeps those addresses:
 * the buffers must stay allocated while it exists. tnsk_plan_destroy waits for
 * the device and frees the plan. Arguments and errors as tnsk_estimate_batch. */
typedef struct tnsk_plan tnsk_plan;
tnsk_status tnsk_plan_create(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, const tnsk_params* params,
                             double* const* outs, double* const* per_reps, tnsk_plan** plan);
/* From its second run on, a plan's launch sequence is captured once into a CUDA
 * graph and replayed with one graph launch, when the ctx stream is not the legacy
 * default stream and profiling is off; otherwise (or if capture fails) the
 * kernels are launched one by one. Results are the same either way. */
tnsk_status tnsk_plan_run(tnsk_ctx* ctx, tnsk_plan* plan);
tnsk_status tnsk_plan_destroy(tnsk_plan* plan);

/* Method-1 estimate that allocates no device memory (the paper has no
 * counterpart; this is a deployment variant of tnsk_estimate).
 * For callers that cannot call cudaMalloc: plugins whose host application owns
 * every allocation, or uses that must not grow device memory after start-up.
 * Needs no ctx. Runs the same kernels as tnsk_estimate with TNSK_GENERAL and
 * TNSK_PREC_FP32 on `cuda_stream` (NULL = legacy default stream) of the current
 * device, with all scratch in one fixed 16 MiB device array inside the library
 * (held by every GPU that loads the library until the process exits).
 * net, params: as for tnsk_estimate (hyperedges get WLOG 1's copy tensors, which
 * are not stored); params->method must be TNSK_GENERAL and params->prec
 * TNSK_PREC_FP32 (else TNSK_ERR_UNSUPPORTED). out, per_rep: device buffers as for
 * tnsk_estimate (per_rep may be NULL).
 * Errors: TNSK_ERR_INVALID / _UNSUPPORTED as tnsk_estimate; TNSK_ERR_UNSUPPORTED
 * also when the call would need more than the 16 MiB of scratch; TNSK_ERR_CUDA
 * when a launch or copy fails. There is no error text.
 * The first call on a device looks up the array and fills its FFT twiddles with
 * a synchronous copy. Every call reuses the same array (each device has its own),
 * so calls on one device whose GPU work overlaps, from two streams or two host
 * threads, race: order them on one stream. */
/* Scatter schedule of a plan (row a2's work items: chunks of a tensor's entries x
 * batches of its reps, one CTA each), per scatter list l = c + 4 k, c the tensor's
 * order class (order <= 2, <= 4, <= 6, above) and k its kernel (0: the FP32 / FP64
 * atomic kernel, 1: the fixed-point kernel with 16-byte loads, 2: the fixed-point
 * kernel with single loads, 3: the fixed-point kernel over whole fibers of a short
 * contracted last mode):
 *   rep_cap[l]     most reps one work item sketches in one pass over its entries
 *                  (0 = default: 32 with privatised bins, 16 without; values above
 *                  those are clamped to them and to what fits in shared memory);
 *   chunk_scale[l] entries per work item as a multiple of the default chunk (0 or 1 =
 *                  default; tensors whose tables are staged per chunk keep 1).
 * Any schedule gives the same estimates up to FP32 rounding order. */
#define TNSK_SCATTER_LISTS 16
typedef struct {
    int32_t rep_cap[TNSK_SCATTER_LISTS];
    int32_t chunk_scale[TNSK_SCATTER_LISTS];
} tnsk_schedule;

/* Autotuner of the scatter schedule of a batch (the arguments of tnsk_estimate_batch
 * without outputs): plans the batch under each candidate (rep_cap in {8, 16, 32} x
 * chunk_scale in {1, 2, 4}, applied to every list), runs each list's scatter launch
 * `trials` times (1..64) on the ctx stream inside the ctx's scratch (CUDA events;
 * the scratch's contents are overwritten), and writes to *sched, per list, the
 * candidate with the least mean time. ms_default / ms_tuned (may be NULL) receive the
 * summed per-launch scatter time of the default schedule and of the chosen one.
 * Synchronous. Errors as tnsk_estimate_batch; TNSK_ERR_INVALID for trials outside
 * 1..64 or a NULL sched. */
tnsk_status tnsk_autotune(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, const tnsk_params* params,
                          int32_t trials, tnsk_schedule* sched, double* ms_default, double* ms_tuned);
/* tnsk_plan_create with a scatter schedule (sched NULL: the default one). */
tnsk_status tnsk_plan_create_scheduled(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets,
                                       const tnsk_params* params, double* const* outs, double* const* per_reps,
                                       const tnsk_schedule* sched, tnsk_plan** plan);

/* The last TNSK_PREC_AUTO estimate on this ctx: reps recomputed in FP64 and the
 * largest relative rounding bound of a per-rep value (see TNSK_PREC_AUTO); 0 and 0
 * before the first. Either pointer may be NULL. */
tnsk_status tnsk_auto_report(tnsk_ctx* ctx, int32_t* fp64_reps, double* max_rel_bound);

tnsk_status tnsk_estimate_static(const tnsk_network* net, const tnsk_params* params, double* out, double* per_rep,
                                 void* cuda_stream);

/* Measurement aid (not part of the method): the rate of FP32 shared-memory
 * atomic adds to random bins (1024 bins x 8 per CTA, 512 threads, four CTAs per
 * SM over all SMs: full occupancy), the ceiling of privatised scatter-add. Runs on the ctx
 * stream, waits for it, and writes updates per second to *updates_per_s. */
tnsk_status tnsk_probe_shared_atomics(tnsk_ctx* ctx, double* updates_per_s);
/* The same for 32-bit integer shared-memory adds whose result is unused (the update
 * of the fixed-point method-1 scatter, TNSK_PREC_FP32): updates per second. */
tnsk_status tnsk_probe_shared_int_adds(tnsk_ctx* ctx, double* updates_per_s);

/* ---- Exact contraction of pairs of tensors (the normalisations of Sec. 4.1:
 * group two tensors into one with their shared contractions summed exactly; a
 * cyclic ladder of two tensor trains becomes an acyclic chain this way). For each
 * job: out[i] = sum over the shared indices of A[...] * B[...], where the shared
 * modes are the pairs (a_modes[j], b_modes[j]), j < n_shared (equal dims); the
 * other modes of A (in order), then of B (in order), are the free modes
 * 0 .. n_free - 1, and output mode i is free mode out_perm[i] (out_perm NULL =
 * identity). out: device FP32, row-major, caller-owned; A, B: device tensors
 * (FP32 / FP64 / BF16). FP32 products summed in FP32.
 * tnsk_pairs_create validates the n jobs (n <= 65535) and uploads their
 * descriptors once (device memory owned by the handle); each tnsk_pairs_run
 * enqueues one launch for all of them on the ctx stream (new data in the same
 * buffers is picked up). tnsk_contract_pairs = create + run + wait + destroy.
 * Errors: TNSK_ERR_INVALID for NULL pointers, bad modes (out of range, repeated,
 * unequal dims) or a bad permutation; TNSK_ERR_UNSUPPORTED above 2^31 output
 * entries or 2^20 shared index combinations per job. */
typedef struct {
    const tnsk_tensor* A;
    const tnsk_tensor* B;
    int32_t n_shared;
    const int32_t* a_modes;
    const int32_t* b_modes;
    const int32_t* out_perm;
    float* out;
} tnsk_pair_job;
typedef struct tnsk_pairs tnsk_pairs;
tnsk_status tnsk_pairs_create(tnsk_ctx* ctx, int32_t n, const tnsk_pair_job* jobs, tnsk_pairs** pairs);
tnsk_status tnsk_pairs_run(tnsk_ctx* ctx, tnsk_pairs* pairs);
tnsk_status tnsk_pairs_destroy(tnsk_pairs* pairs);
/* Makes every later tnsk_plan_run of `plan` run `pairs` (as tnsk_pairs_run) on the ctx
 * stream ahead of the plan's method-2 work, while the plan's method-1 work runs on the
 * ctx's second stream: pair contractions that produce method-2 tensors (a merged
 * chain) then overlap the method-1 sketches instead of preceding the whole run. The
 * pairs' outputs must not be read by the plan's method-1 networks. NULL detaches. The
 * handle must stay alive while the plan runs it; a captured run sequence is captured
 * again on the next run. */
tnsk_status tnsk_plan_set_prelude(tnsk_ctx* ctx, tnsk_plan* plan, tnsk_pairs* pairs);
tnsk_status tnsk_contract_pairs(tnsk_ctx* ctx, int32_t n, const tnsk_pair_job* jobs);

/* ---- Learned sketch-size predictor (the paper has no counterpart: it sizes m
 * by its variance bounds). A multilayer perceptron TNSK_MLP_FEATURES -> 128 ->
 * 128 -> 128 -> 1, GELU (x Phi(x)) after each hidden layer, maps the features of
 * a network at sketch size m and R reps (tnsk_features) to log10 of the relative
 * error |y - tc| / |tc| of the method-1 estimate; trained by mean squared error
 * and Adam (FP32) on samples the caller measures, evaluated in FP32 or with BF16
 * operands (FP32 accumulation). Parameters: per layer W [n_out][n_in] row-major,
 * then b [n_out], layers in order (tnsk_mlp_num_params floats); inputs are
 * standardised per feature with mu, sigma (norm = mu[F] then sigma[F]) taken from
 * the last training set. All X / y / grad pointers are device FP32, row-major
 * [n][TNSK_MLP_FEATURES]. Calls run on the ctx stream; get, save, loss_grad and
 * train return after the device work. */
#define TNSK_MLP_FEATURES 9
typedef struct tnsk_mlp tnsk_mlp;
tnsk_status tnsk_mlp_num_params(int64_t* n);
/* W ~ U(-a, a), a = sqrt(6 / n_in), b = 0 (seeded); identity standardisation. */
tnsk_status tnsk_mlp_create(tnsk_ctx* ctx, uint64_t seed, tnsk_mlp** mlp);
tnsk_status tnsk_mlp_destroy(tnsk_mlp* mlp);
/* host copies: theta[tnsk_mlp_num_params], norm[2 * TNSK_MLP_FEATURES] */
tnsk_status tnsk_mlp_get(tnsk_mlp* mlp, float* theta, float* norm);
tnsk_status tnsk_mlp_set(tnsk_ctx* ctx, tnsk_mlp* mlp, const float* theta, const float* norm);
/* Mean squared error of the n rows and its gradient (device, tnsk_mlp_num_params
 * floats; may be NULL) at the current parameters; *loss on the host. n <= 2^24. */
tnsk_status tnsk_mlp_loss_grad(tnsk_ctx* ctx, tnsk_mlp* mlp, const float* X, const float* y, int64_t n, float* grad,
                               double* loss);
/* Sets the standardisation from X, then `epochs` passes of Adam (lr, beta 0.9 /
 * 0.999, eps 1e-8) over minibatches of `batch` rows in a seeded random order;
 * *final_loss (may be NULL) = the mean squared error over all n rows after. */
tnsk_status tnsk_mlp_train(tnsk_ctx* ctx, tnsk_mlp* mlp, const float* X, const float* y, int64_t n, int32_t epochs,
                           int32_t batch, float lr, uint64_t seed, double* final_loss);
/* y[i] = predicted log10 relative error of row i; bf16 != 0: BF16 operands. */
tnsk_status tnsk_mlp_predict(tnsk_ctx* ctx, tnsk_mlp* mlp, const float* X, int64_t n, float* y, int32_t bf16);
/* Binary file of this library ("TNSKMLP1", shape, norm, theta); load checks the shape. */
tnsk_status tnsk_mlp_save(tnsk_mlp* mlp, const char* path);
tnsk_status tnsk_mlp_load(tnsk_ctx* ctx, tnsk_mlp* mlp, const char* path);
/* Features (host float[TNSK_MLP_FEATURES]) of a network at params->m and
 * params->reps: p, t, cycle rank t - p + components, log2 of the largest and the
 * mean log2 of the contraction dims, mean and standard deviation over tensors of
 * ln ||X_k||_F (computed on the device), log2 m, log2 R. */
tnsk_status tnsk_features(tnsk_ctx* ctx, const tnsk_network* net, const tnsk_params* params, float* features);
/* Sets inout->m to the smallest 2^6 .. 2^16 whose predicted relative error at
 * inout->reps is <= target_err (*predicted_err, may be NULL, gets it). The
 * predicted error is the 90% quantile of one estimate's relative error: the
 * predictor's expected log10 error, shifted by the log10 |Z| statistics of a
 * normal error (10^pred / 0.3224). With
 * mlp == NULL, or for TNSK_ACYCLIC, the paper's variance bound with delta = 0.1
 * decides instead: m R >= 3^t / (eps^2 delta) (general) or 32 t / (eps^2 delta)
 * (acyclic). TNSK_ERR_UNREACHABLE (inout unchanged, *predicted_err = the best
 * candidate's) when no candidate meets the target. */
tnsk_status tnsk_choose_params(tnsk_ctx* ctx, const tnsk_network* net, double target_err, tnsk_mlp* mlp,
                               tnsk_params* inout, double* predicted_err);

/* Fault injection for tests (the paper has no counterpart): what = 1 makes the next
 * launch sequence of this ctx run method 2's TMA-fed tensor-core products (the FP32
 * streaming kernel and the BF16 kernel) with producers that issue no loads, so every
 * consumer's bounded wait (at most about 2^31 SM clock cycles) runs out and records
 * TNSK_ERR_TIMEOUT for tnsk_sync; no copy or MMA is left in flight and the ctx stays
 * usable. One-shot (cleared by that launch sequence); what = 0 clears it. Plans
 * replayed from a CUDA graph keep the setting they were captured with. Errors:
 * TNSK_ERR_INVALID for a NULL ctx or another value. */
tnsk_status tnsk_debug_inject(tnsk_ctx* ctx, int32_t what);

/* Parameters for B networks at once (the library's sizing policy; the paper sizes m
 * by its variance bounds only). For every network, the cheapest (m, R) with m in
 * 2^6 .. 2^16 and R in {16, 32, 64} (the normal quantile of a mean of fewer, heavy-
 * tailed repetitions is not trusted), the cost being Theorem 1's work per
 * repetition times R, R (sum_k q_k N_k + p m log2 m), whose predicted relative error
 * |y - tc| / |tc| (90% quantile) is at most target_err:
 *   1. from the learned predictor (TNSK_GENERAL networks, mlp not NULL; how[b] = 0);
 *   2. else, with pilot_reps >= 2, from a pilot: pilot_reps repetitions at m = 2^12
 *      of all such networks in one batch (repetitions rep0 = 2^20 on, apart from the
 *      estimate's), whose sample variance s^2, taken one standard error up
 *      (s^2 (1 + sqrt(2 / (pilot_reps - 1)))), scales as 1/m per repetition (both
 *      variance lemmas) and 1/R for the mean: 1.6449 sqrt(s^2 2^12 / (m R)) / |mean|
 *      (how[b] = 1);
 *   3. else the cheapest candidate, m = 2^6 and R = 16, flagged how[b] = 2 with
 *      predicted_err[b] the best candidate's (no affordable work meets the target; the
 *      caller decides whether a larger estimate is worth it).
 * inout[b]: m, reps and groups (1) are set, other fields kept. predicted_err, how: host
 * arrays [B]. Runs the pilot on the ctx stream and waits for it. Errors: as
 * tnsk_estimate for a network; TNSK_ERR_INVALID for bad arguments (pilot_reps 1 or
 * above 4096); TNSK_ERR_UNSUPPORTED for TNSK_CROSSCORR. */
tnsk_status tnsk_choose_params_batch(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, double target_err,
                                     tnsk_mlp* mlp, int32_t pilot_reps, tnsk_params* inout, double* predicted_err,
                                     int32_t* how);

/* Parameters for B networks for the most estimates within target_err per unit of work
 * over the batch (a throughput policy of the library; the paper sizes m by its variance
 * bounds only). The candidates, their cost R (sum_k q_k N_k + p m log2 m) and the
 * sources of prediction are those of tnsk_choose_params_batch; both policies model one
 * estimate's relative error as sigma |Z| (Z standard normal; from the predictor,
 * log10 sigma = prediction + 0.2757, since E log10 |Z| = -0.2757; from the pilot,
 * sigma = s / |mean| with s^2 as there), so a candidate meets the target with chance
 * P = erf(target_err / (sigma sqrt 2)). The choice maximises sum_b P_b / sum_b cost_b:
 * Dinkelbach's iteration, each network taking the candidate that maximises
 * P - lambda cost with lambda the batch's current ratio, until lambda stops rising.
 * A network is sized where the predictor covers it (how[b] = 0), else by the pilot when
 * pilot_reps >= 2 (how[b] = 1; networks with a prediction are not piloted); where its
 * chosen chance is below 1/2 it is flagged how[b] = 2 (meeting the target costs more
 * than it returns at the batch's rate), its candidate still the one chosen.
 * predicted_err[b]: the chosen candidate's 90% quantile, 1.6449 sigma (1e300 where
 * nothing predicts it). inout, predicted_err, how, waits and errors: as
 * tnsk_choose_params_batch. */
tnsk_status tnsk_choose_params_rate(tnsk_ctx* ctx, int32_t B, const tnsk_network* nets, double target_err,
                                    tnsk_mlp* mlp, int32_t pilot_reps, tnsk_params* inout, double* predicted_err,
                                    int32_t* how);

/* Wait for the ctx's stream; returns the first deferred device error, if any. */
tnsk_status tnsk_sync(tnsk_ctx* ctx);

const char* tnsk_status_string(tnsk_status s);
/* Text of the last error on this ctx ("" if none). */
const char* tnsk_last_error(tnsk_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* TNSK_H */
