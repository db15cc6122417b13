// plan.cu -- validation of a network against the statement of the problem
// (Sec. 1 Def. "Tensor contraction": u != v and n_u = n_v for every (u, v) in E;
// Sec. 4.1 WLOG 1: a mode is part of at most one contraction) and the layout of
// one batch's descriptors and scratch.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <limits>
#include <mutex>

#include "plan.cuh"

namespace tnsk {

namespace {

constexpr int64_t kMaxNumel = (int64_t)1 << 40;
constexpr size_t kScatterSmemBudget = 96 * 1024;

// Largest m whose FFT runs inside one CTA's shared memory (block kernels, method 2's
// composition); method 1 goes further (2^16) with the two-pass large-m kernels.
int max_log2m_for(bool fp64) { return fp64 ? 13 : 14; }
constexpr int kMaxLog2mLarge = 16;

template <class T>
size_t stage(std::vector<unsigned char>& buf, const std::vector<T>& v) {
    size_t at = (buf.size() + 255) & ~(size_t)255;
    buf.resize(at + v.size() * sizeof(T));
    if (!v.empty()) std::memcpy(buf.data() + at, v.data(), v.size() * sizeof(T));
    return at;
}

int ilog2(int64_t x) {
    int l = 0;
    while (((int64_t)1 << l) < x) ++l;
    return l;
}

// Offset (in words) of T_{l,j} side s inside a node's T block; levels are
// stored from l = qt down to 2, level l holding l/2 pairs.
int64_t ts_offset(int qt, int l, int j, int s, int64_t m) {
    int64_t before = 0;
    for (int ll = qt; ll > l; ll >>= 1) before += ll / 2;
    return ((before + j) * 2 + s) * m;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        cudaGetLastError();
    });
    return fn;
}

}  // namespace

bool tensor_maps_available() { return encoder() != nullptr; }

// Row-major FP32 matrix [rows][cols] (cols % 4 == 0, 16-byte aligned) as 2-D
// TMA boxes of 32 columns x box_rows rows, 128-byte swizzle, zero fill outside; with
// bf16, a BF16 matrix (cols % 8 == 0) in boxes of 64 columns (128-byte rows).
static bool encode_rowmajor(void* out, const void* base, int64_t rows, int64_t cols, int box_rows,
                            bool bf16 = false) {
    EncodeTiledFn fn = encoder();
    if (!fn) return false;
    CUtensorMap tm;
    cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)cols * (bf16 ? 2 : 4)};
    cuuint32_t box[2] = {bf16 ? 64u : 32u, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(&tm, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                    const_cast<void*>(base), gdim, gstride, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    std::memcpy(out, &tm, sizeof(tm));
    return true;
}

tnsk_status finalize_plan(BatchPlan& P, unsigned char* base, std::string& err) {
    if (P.m2.tmap_jobs.empty()) return TNSK_OK;
    const M2Node* nodes = (const M2Node*)(P.host_desc.data() + (P.m2.nodes_off - P.desc_off));
    const M2Net* nets = (const M2Net*)(P.host_desc.data() + (P.m2.nets_off - P.desc_off));
    unsigned char* maps = P.host_desc.data() + (P.m2.tmaps_off - P.desc_off);
    const float* ws = (const float*)(base + P.m2.ws_off);
    for (size_t i = 0; i < P.m2.tmap_jobs.size(); ++i) {
        const M2Node& nd = nodes[P.m2.tmap_jobs[i].first];
        // 0: X, 1: V^T hi, 2: V^T lo (FP32); 3: X, 4 .. 6: the three parts of V^T (BF16);
        // 7, 8: V^T hi, lo of a grouped node viewed as [R cols / 32][32], boxes of 128 rows
        const int what = P.m2.tmap_jobs[i].second;
        const int64_t R = nets[nd.net].R;
        bool ok;
        if (what == 0)
            ok = encode_rowmajor(maps + i * 128, nd.data, nd.npar, nd.cols, 128);
        else if (what <= 2)
            ok = encode_rowmajor(maps + i * 128, ws + nd.v_off + (what - 1) * R * nd.cols, R, nd.cols, 64);
        else if (what == 3)
            ok = encode_rowmajor(maps + i * 128, nd.data, nd.npar, nd.cols, 128, true);
        else if (what >= 7)
            ok = encode_rowmajor(maps + i * 128, ws + nd.v_off + (what - 7) * R * nd.cols, R * nd.cols / 32, 32, 128);
        else
            ok = encode_rowmajor(maps + i * 128, (const unsigned char*)(ws + nd.v_off) + (what - 4) * R * nd.cols * 2,
                                 R, nd.cols, 64, true);
        if (!ok) {
            err = "tensor-map encoding failed";
            return TNSK_ERR_CUDA;
        }
    }
    return TNSK_OK;
}

// Grouped tensors run the tensor-core kernel that forms their entries where its layout
// rules hold (column fast index a multiple of 32, B factor within 60 KiB, tensor maps);
// otherwise, with all four factor dims at most 32, the factored SIMT product
// (m2_rung_fact.cu), measured slower than the tensor-core kernel at dims 32.
static bool rung_small(const tnsk_rung& g) { return g.a <= 32 && g.b <= 32 && g.c <= 32 && g.d <= 32; }

tnsk_status validate(const tnsk_network& net, const tnsk_params& prm, NetInfo& I, std::string& why, bool zero_ok,
                     const char* diag) {
    if (net.p < 1 || !net.X) {
        why = "need p >= 1 tensors";
        return TNSK_ERR_INVALID;
    }
    const bool fp64 = prm.prec == TNSK_PREC_FP64;
    if (prm.prec == TNSK_PREC_AUTO) {
        why = "TNSK_PREC_AUTO is taken by tnsk_estimate only (one network, method 1, no open legs)";
        return TNSK_ERR_UNSUPPORTED;
    }
    if (prm.prec != TNSK_PREC_FP32 && prm.prec != TNSK_PREC_BF16 && prm.prec != TNSK_PREC_FP64) {
        why = "unknown precision";
        return TNSK_ERR_INVALID;
    }
    if (prm.method != TNSK_GENERAL && prm.method != TNSK_ACYCLIC && prm.method != TNSK_CROSSCORR) {
        why = "unknown method";
        return TNSK_ERR_INVALID;
    }
    if (prm.m < 1 || (prm.m & (prm.m - 1))) {
        why = "sketch size m must be a power of two >= 1";
        return TNSK_ERR_UNSUPPORTED;
    }
    I.log2m = ilog2(prm.m);
    if (I.log2m > (is_m1(prm.method) ? kMaxLog2mLarge : max_log2m_for(fp64))) {
        why = is_m1(prm.method) ? "sketch size m above 2^16"
                                         : "method 2: sketch size m above the single-CTA FFT limit (2^14 FP32, 2^13 FP64)";
        return TNSK_ERR_UNSUPPORTED;
    }
    if (prm.reps < 1 || prm.reps > 65536) {
        why = "reps must be in [1, 65536]";
        return TNSK_ERR_INVALID;
    }
    if (prm.rep0 < 0) {
        why = "rep0 must be >= 0";
        return TNSK_ERR_INVALID;
    }
    if (prm.groups < 1 || prm.groups > 64 || prm.reps % prm.groups != 0) {
        why = "groups must divide reps and be in [1, 64]";
        return TNSK_ERR_INVALID;
    }
    I.p = net.p;
    I.mode_off.assign(I.p + 1, 0);
    for (int k = 0; k < I.p; ++k) {
        const tnsk_tensor& X = net.X[k];
        if (X.order < 0) {
            why = "negative order";
            return TNSK_ERR_INVALID;
        }
        if (X.order > TNSK_MAX_ORDER) {
            why = "tensor order above 12";
            return TNSK_ERR_UNSUPPORTED;
        }
        if (X.order > 0 && !X.dims) {
            why = "null dims";
            return TNSK_ERR_INVALID;
        }
        if (X.dtype != TNSK_F64 && X.dtype != TNSK_F32 && X.dtype != TNSK_BF16) {
            why = "unknown dtype";
            return TNSK_ERR_INVALID;
        }
        I.mode_off[k + 1] = I.mode_off[k] + X.order;
    }
    I.q = I.mode_off[I.p];
    I.dims.resize(I.q);
    I.tensor_of.resize(I.q);
    I.numel.assign(I.p, 1);
    I.idx32 = true;
    for (int k = 0; k < I.p; ++k) {
        const tnsk_tensor& X = net.X[k];
        const bool is_diag = diag && diag[k];  // never stored: only its n nonzeros are read
        const int64_t max_numel = is_diag ? ((int64_t)1 << 62) : kMaxNumel;
        int64_t n = 1;
        for (int d = 0; d < X.order; ++d) {
            int64_t v = X.dims[d];
            if (v < 0) {
                why = "negative dim";
                return TNSK_ERR_INVALID;
            }
            if (v > std::numeric_limits<int32_t>::max()) {
                why = "dim above 2^31 - 1";
                return TNSK_ERR_UNSUPPORTED;
            }
            I.dims[I.mode_off[k] + d] = v;
            I.tensor_of[I.mode_off[k] + d] = k;
            if (v == 0)
                n = 0;
            else if (n > 0) {
                if (n > max_numel / v) {
                    why = "tensor above 2^40 entries";
                    return TNSK_ERR_UNSUPPORTED;
                }
                n *= v;
            }
        }
        I.numel[k] = n;
        I.rung.push_back(X.rung);
        I.diag.push_back(is_diag ? 1 : 0);
        if (X.rung) {
            I.zero.push_back(0);  // grouped tensor (Sec. 4.1): R((i,j),(k,l)) = sum_s A(i,s,k) B(j,s,l)
            const tnsk_rung& g = *X.rung;
            if (prm.method != TNSK_ACYCLIC || prm.prec == TNSK_PREC_FP64) {
                why = "tensor " + std::to_string(k) + ": grouped (rung) tensors need method 2 in FP32";
                return TNSK_ERR_UNSUPPORTED;
            }
            if (X.order != 2 || X.dtype != TNSK_F32 || X.data || !g.A || !g.B || g.a < 1 || g.s < 1 || g.c < 1 ||
                g.b < 1 || g.d < 1 || X.dims[0] != g.a * g.b || X.dims[1] != g.c * g.d) {
                why = "tensor " + std::to_string(k) +
                      ": a rung tensor is order 2, FP32, data NULL, dims [a*b, c*d], A and B set, sizes >= 1";
                return TNSK_ERR_INVALID;
            }
            const int64_t lim = (int64_t)1 << 31;
            if (g.s > 16 || g.a * g.s * g.c >= lim || g.b * g.s * g.d >= lim || n >= lim) {
                why = "tensor " + std::to_string(k) + ": rung tensor above the kernel's limits (s <= 16, < 2^31 entries)";
                return TNSK_ERR_UNSUPPORTED;
            }
            continue;
        }
        I.zero.push_back(n > 0 && !X.data && (zero_ok || is_diag) ? 1 : 0);
        if (n > 0 && !X.data && !zero_ok && !is_diag) {
            why = "null data for a non-empty tensor";
            return TNSK_ERR_INVALID;
        }
        if (n >= ((int64_t)1 << 32) && !is_diag) I.idx32 = false;
    }
    I.t = net.t;
    if (I.t < 0 || (I.t > 0 && !net.edges)) {
        why = "bad contraction list";
        return TNSK_ERR_INVALID;
    }
    I.edge_of.assign(I.q, -1);
    I.side_of.assign(I.q, 0);
    I.open_pos.assign(I.q, -1);
    I.eoff.assign(I.t + 1, 0);
    for (int e = 0; e < I.t; ++e) {
        int u = net.edges[2 * e], v = net.edges[2 * e + 1];
        if (u < 0 || v < 0 || u >= I.q || v >= I.q || u == v) {
            why = "contraction " + std::to_string(e) + " needs two distinct valid modes";
            return TNSK_ERR_INVALID;
        }
        if (I.dims[u] != I.dims[v]) {
            why = "contraction " + std::to_string(e) + " joins modes of different size";
            return TNSK_ERR_INVALID;
        }
        if (I.edge_of[u] >= 0 || I.edge_of[v] >= 0) {
            why = "a mode in two contractions (a hyperedge: WLOG 1 copy tensors are built for TNSK_GENERAL and "
                  "TNSK_CROSSCORR only)";
            return TNSK_ERR_UNSUPPORTED;
        }
        I.edge_of[u] = e;
        I.side_of[u] = 0;
        I.edge_of[v] = e;
        I.side_of[v] = 1;
        I.eoff[e + 1] = I.eoff[e] + I.dims[u];
    }
    I.L = I.eoff[I.t];
    int n_free = 0;
    for (int g = 0; g < I.q; ++g)
        if (I.edge_of[g] < 0) ++n_free;
    if (net.n_open != n_free || (n_free > 0 && !net.open)) {
        why = "open list must be a permutation of the uncontracted modes";
        return TNSK_ERR_INVALID;
    }
    I.O = 1;
    for (int j = 0; j < net.n_open; ++j) {
        int g = net.open[j];
        if (g < 0 || g >= I.q || I.edge_of[g] >= 0 || I.open_pos[g] >= 0) {
            why = "open list must be a permutation of the uncontracted modes";
            return TNSK_ERR_INVALID;
        }
        I.open_pos[g] = j;
        if (I.dims[g] > 0 && I.O > kMaxNumel / I.dims[g]) {
            why = "output above 2^40 entries";
            return TNSK_ERR_UNSUPPORTED;
        }
        I.O *= I.dims[g];
    }
    I.open_tot.assign(I.p, 1);
    int n_ot = 0;
    for (int k = 0; k < I.p; ++k) {
        int64_t o = 1;
        for (int g = I.mode_off[k]; g < I.mode_off[k + 1]; ++g)
            if (I.edge_of[g] < 0) o *= I.dims[g];
        I.open_tot[k] = o;
        if (o > 1) ++n_ot;
    }
    if (is_m1(prm.method)) {
        if (n_ot > TNSK_MAX_OPEN_TENSORS) {
            why = "open legs on more than 4 tensors";
            return TNSK_ERR_UNSUPPORTED;
        }
        return TNSK_OK;
    }
    // ---- method 2: acyclic, connected, full (Sec. 4.4) ----
    if (net.n_open != 0) {
        why = "the acyclic method takes open legs in tnsk_estimate and tnsk_estimate_batch only (one full estimate "
              "per output entry), not in plans, streams or parameter choices";
        return TNSK_ERR_UNSUPPORTED;
    }
    for (int e = 0; e < I.t; ++e)
        if (I.tensor_of[net.edges[2 * e]] == I.tensor_of[net.edges[2 * e + 1]]) {
            why = "a contraction inside one tensor is a cycle for the acyclic method";
            return TNSK_ERR_CYCLIC;
        }
    if (I.t > I.p - 1) {
        why = "more contractions than a tree has: the network has a cycle";
        return TNSK_ERR_CYCLIC;
    }
    if (I.t < I.p - 1) {
        why = "the network is not connected";
        return TNSK_ERR_UNSUPPORTED;
    }
    if (prm.root >= I.p || prm.root < -1) {
        why = "root out of range";
        return TNSK_ERR_INVALID;
    }
    int root = prm.root;
    if (root < 0) {
        root = 0;
        for (int k = 1; k < I.p; ++k)
            if (I.numel[k] < I.numel[root]) root = k;
    }
    I.root = root;
    I.parent.assign(I.p, -1);
    I.parent_mode.assign(I.p, -1);
    I.parent_edge.assign(I.p, -1);
    I.child.assign(I.p, {});
    I.child_mode.assign(I.p, {});
    I.child_edge.assign(I.p, {});
    std::vector<int> seen(I.p, 0), order;
    order.push_back(root);
    seen[root] = 1;
    for (size_t h = 0; h < order.size(); ++h) {
        int k = order[h];
        for (int g = I.mode_off[k]; g < I.mode_off[k + 1]; ++g) {
            int e = I.edge_of[g];
            if (e == I.parent_edge[k]) continue;
            int other = net.edges[2 * e] == g ? net.edges[2 * e + 1] : net.edges[2 * e];
            int l = I.tensor_of[other];
            if (seen[l]) {
                why = "two contractions between one pair of tensors (merge them, WLOG 3)";
                return TNSK_ERR_CYCLIC;
            }
            seen[l] = 1;
            I.child[k].push_back(l);
            I.child_mode[k].push_back(g - I.mode_off[k]);
            I.child_edge[k].push_back(e);
            I.parent[l] = k;
            I.parent_edge[l] = e;
            I.parent_mode[l] = other - I.mode_off[l];
            order.push_back(l);
        }
    }
    if ((int)order.size() != I.p) {
        why = "the network is not connected";
        return TNSK_ERR_UNSUPPORTED;
    }
    I.height.assign(I.p, 0);
    for (int h = (int)order.size() - 1; h >= 0; --h) {
        int k = order[h];
        if ((int)I.child[k].size() > TNSK_MAX_SLOTS) {
            why = "a tensor with more than 16 children";
            return TNSK_ERR_UNSUPPORTED;
        }
        for (int l : I.child[k]) I.height[k] = std::max(I.height[k], I.height[l] + 1);
    }
    I.max_height = I.height[root];
    return TNSK_OK;
}

namespace {
struct PlanLists {
    std::vector<TabReq> reqs;
    std::vector<M1Tensor> m1t;
    std::vector<M1Net> m1n;
    std::vector<M1Work> m1w;
    std::vector<OpenMode> opens;
    std::vector<int2> m1items;
    std::vector<int2> m1warp[M1Plan::kWarpSlots];
    std::vector<CombineItem> comb;
    std::vector<M2Node> m2nodes;
    std::vector<M2Net> m2n;
    std::vector<int4> lfft, lprod, mfft, mprod;
    std::vector<M1Diag> diags;
    std::vector<M1RowSort> rsorts;
    std::vector<M1RowItem> ritems;
    std::vector<M1Work> m1w_cls[M1Plan::kScatterLists];
    std::vector<M2Item> m2items;
};

// This thread's lists, emptied (capacity kept).
PlanLists& plan_lists() {
    static thread_local PlanLists L;
    L.reqs.clear();
    L.m1items.clear();
    L.m1t.clear();
    L.m1n.clear();
    L.m1w.clear();
    L.opens.clear();
    for (auto& v : L.m1warp) v.clear();
    L.comb.clear();
    L.m2nodes.clear();
    L.m2n.clear();
    for (auto* v : {&L.lfft, &L.lprod, &L.mfft, &L.mprod}) v->clear();
    L.diags.clear();
    L.rsorts.clear();
    L.ritems.clear();
    for (auto& v : L.m1w_cls) v.clear();
    L.m2items.clear();
    return L;
}

// A staged descriptor block that has been uploaded, kept for the thread's next plan.
thread_local std::vector<unsigned char> g_desc_pool;

void take_desc_buffer(std::vector<unsigned char>& H) {
    if (H.capacity() < g_desc_pool.capacity()) H.swap(g_desc_pool);
    H.clear();
}
}  // namespace

void recycle_host_desc(std::vector<unsigned char>& H) {
    if (H.capacity() > g_desc_pool.capacity()) {
        H.clear();
        g_desc_pool.swap(H);
    }
}

tnsk_status plan_batch(const std::vector<NetInfo>& infos, const tnsk_network* nets, const tnsk_params* params,
                       double* const* outs, double* const* per_reps, bool fp64, bool sketch_only, BatchPlan& P,
                       std::string& err, const tnsk_schedule* sched, const int64_t* rep_stride) {
    const int B = (int)infos.size();
    const size_t acc = fp64 ? sizeof(double) : sizeof(float);
    // The descriptor lists live in per-thread vectors that keep their capacity from one
    // plan to the next: a batch of large-m networks stages megabytes of items, and fresh
    // vectors grown by doubling spent most of the planning time in page faults.
    PlanLists& L = plan_lists();
    std::vector<TabReq>& reqs = L.reqs;
    std::vector<M1Tensor>& m1t = L.m1t;
    std::vector<M1Net>& m1n = L.m1n;
    std::vector<M1Work>& m1w = L.m1w;
    std::vector<OpenMode>& opens = L.opens;
    std::vector<int2>& m1items = L.m1items;
    std::vector<int2>* m1warp = L.m1warp;
    std::vector<CombineItem>& comb = L.comb;
    std::vector<M2Node>& m2nodes = L.m2nodes;
    std::vector<M2Net>& m2n = L.m2n;
    int64_t tab_words = 0, yrep_n = 0, xs_n = 0, spec_n = 0, sexp_n = 0, lspec_n = 0;
    // large-m method 1: (net, rep, sketch), (net, rep, first bin, bins)
    std::vector<int4>& lfft = L.lfft;
    std::vector<int4>& lprod = L.lprod;
    // mid-m closed networks: the same item forms
    std::vector<int4>& mfft = L.mfft;
    std::vector<int4>& mprod = L.mprod;
    int mid_max_log2m = 0;
    std::vector<M1Diag>& diags = L.diags;      // diagonal copy tensors (WLOG 1)
    std::vector<M1RowSort>& rsorts = L.rsorts;  // row-sorted sketches of large tensors
    std::vector<M1RowItem>& ritems = L.ritems;
    int64_t rs_words = 0;           // their sorted-row scratch (uint32 words)
    int64_t ws_x = 0, ws_w = 0, ws_r = 0, ws_v = 0;  // method-2 workspace parts (elements)
    int64_t ws_c = 0;  // prepared factors of grouped tensors on the factored tensor-core product
    const bool tma = tensor_maps_available();
    int max_log2m1 = 0, max_log2m2 = 0;
    std::vector<M1Work>* m1w_cls = L.m1w_cls;
    struct PendingItem {
        int h, kind;
        M2Item it;
    };
    std::vector<PendingItem> pend;
    // method-2 node-local offsets are finalised after the x / r / V totals are known
    struct M2Fix {
        size_t node;
        int64_t x, w, r, v, src;
        int64_t c;     // prepared factors (M2_GEMM_RUNGT), -1 none
        int src_kind;  // 0 none, 1 r part, 2 x part
        int64_t child_x[TNSK_MAX_SLOTS];
    };
    std::vector<M2Fix> fixes;

    for (int b = 0; b < B; ++b) {
        const NetInfo& I = infos[b];
        const tnsk_network& N = nets[b];
        const tnsk_params& pr = params[b];
        const int64_t m = pr.m;
        const uint32_t mask = (uint32_t)(m - 1);
        const int R = pr.reps;
        if (is_m1(pr.method)) {
            M1Net nb{};
            nb.m = m;
            nb.log2m = I.log2m;
            nb.R = R;
            nb.groups = pr.groups;
            nb.L = I.L;
            nb.tab_off = tab_words;
            nb.O = I.O;
            nb.y_off = yrep_n;
            nb.t0 = (int)m1t.size();
            nb.p = I.p;
            nb.open0 = (int)opens.size();
            nb.n_open = N.n_open;
            nb.out = outs ? outs[b] : nullptr;
            nb.per_rep = per_reps ? per_reps[b] : nullptr;
            const int64_t K = m == 1 ? 1 : m / 2 + 1;
            int64_t xacc = 0, sacc = 0, eacc = 0;
            std::vector<int> slot_of(I.p, -1);
            for (int k = 0; k < I.p; ++k) {
                M1Tensor T{};
                T.data = N.X[k].data;
                T.numel = I.numel[k];
                T.O = I.open_tot[k];
                T.xoff = xacc;
                xacc += T.O * m;
                if (T.O > 1) {
                    slot_of[k] = nb.n_ot;
                    nb.ot[nb.n_ot++] = (int)m1t.size();
                    T.soff = sacc;
                    T.eoff = eacc;
                    sacc += T.O * K;
                    eacc += T.O;
                } else {
                    T.soff = -1;
                    T.eoff = -1;
                }
                T.dtype = N.X[k].dtype;
                T.order = N.X[k].order;
                T.net = (int)m1n.size();
                int64_t ost = 1;
                for (int d = T.order - 1; d >= 0; --d) {
                    int g = I.mode_off[k] + d;
                    T.dims[d] = (int32_t)I.dims[g];
                    if (I.edge_of[g] >= 0) {
                        T.tab[d] = (int32_t)I.eoff[I.edge_of[g]];
                        // method 1: the second mode of each contraction takes C'; the
                        // cross-correlation chain: every mode of a conjugated tensor
                        T.comp[d] = pr.method == TNSK_CROSSCORR ? ((I.p - 1 - k) & 1) : I.side_of[g];
                        T.ostride[d] = 0;
                        T.n_ctr++;
                    } else {
                        T.tab[d] = -1;
                        T.comp[d] = 0;
                        T.ostride[d] = ost;
                        ost *= I.dims[g];
                    }
                }
                m1t.push_back(T);
            }
            nb.X = xacc;
            nb.x_off = sketch_only ? 0 : xs_n;
            nb.spec_per_rep = sacc;
            nb.spec_off = spec_n;
            nb.exp_per_rep = eacc;
            nb.exp_off = sexp_n;
            // output modes: row-major over the open list
            int64_t ostr = 1;
            std::vector<OpenMode> om(N.n_open);
            for (int j = N.n_open - 1; j >= 0; --j) {
                int g = N.open[j];
                int k = I.tensor_of[g];
                int64_t ts = 1;
                for (int g2 = g + 1; g2 < I.mode_off[k + 1]; ++g2)
                    if (I.edge_of[g2] < 0) ts *= I.dims[g2];
                om[j].ostride = ostr;
                om[j].tstride = ts;
                om[j].dim = (int32_t)I.dims[g];
                om[j].slot = slot_of[k];
                ostr *= I.dims[g];
            }
            opens.insert(opens.end(), om.begin(), om.end());
            // tables: one count sketch per contraction and rep (Alg. 1 first loop)
            for (int e = 0; e < I.t; ++e) {
                TabReq q{};
                q.seed = pr.seed;
                q.rep_base = pr.rep0;
                q.tid = tid_m1_edge(e);
                q.n = I.eoff[e + 1] - I.eoff[e];
                q.out_off = tab_words + I.eoff[e];
                q.rep_stride = I.L;
                q.R = R;
                q.mask = mask;
                if (q.n > 0) reqs.push_back(q);
            }
            tab_words += (int64_t)R * I.L;
            // scatter work: chunks of each tensor x batches of reps
            for (int k = 0; k < I.p; ++k) {
                const M1Tensor& T = m1t[nb.t0 + k];
                if (I.diag[k] && T.numel > 0) diags.push_back(M1Diag{nb.t0 + k, (int)m1n.size(), I.dims[I.mode_off[k]]});
                if (T.numel == 0 || T.O == 0 || I.zero[k]) continue;  // all-zero tensors add nothing
                // Large FP32 tensors (far beyond L2) with a contracted leading mode, at most
                // two reps: the row-sorted form, one pass over the tensor per rep
                // (m1_rowsort.cu); more reps share one pass of the entry scatter
                if (!fp64 && !I.diag[k] && T.dtype == TNSK_F32 && T.O == 1 && T.order >= 2 && T.tab[0] >= 0 &&
                    T.numel >= ((int64_t)1 << 24) && T.dims[0] >= 1024 && T.dims[0] <= (1 << 16) &&
                    m <= (1 << 14) && R <= 2) {
                    bool all_ctr = true;
                    for (int d = 1; d < T.order; ++d) all_ctr = all_ctr && (T.tab[d] >= 0 || T.dims[d] == 1);
                    const int64_t rl = T.numel / T.dims[0];
                    // four columns per lane: 16-byte loads of every row
                    if (all_ctr && rl >= 2048 && (rl & 3) == 0 && ((uintptr_t)T.data & 15) == 0) {
                        const int64_t strips = (rl + 2047) / 2048;
                        for (int r = 0; r < R; ++r) {
                            rsorts.push_back(M1RowSort{nb.t0 + k, (int)m1n.size(), r, (int)strips, rs_words});
                            rs_words += (T.dims[0] + 63) / 64 * 64;
                        }
                        P.m1.rs_max_m = std::max<int64_t>(P.m1.rs_max_m, m);
                        continue;
                    }
                }
                int64_t TT = 0;
                for (int d = 0; d < T.order; ++d)
                    if (T.tab[d] >= 0) TT += T.dims[d];
                // tables above 8 KiB per rep: staged per chunk when the index ranges a chunk
                // of privatised bins touches fit (ltab: a large tensor's leading modes cover
                // a few indices per chunk), else read from global memory (L2)
                const size_t bin_b = (size_t)T.O * m * acc;
                bool gtab = TT > 2048, ltab = false;
                int64_t TTl = TT;
                if (gtab && T.numel * 4 >= T.O * m) {
                    const int64_t CHl = std::max<int64_t>(8192, 32 * T.O * m);
                    int64_t P = 1, tl = 0;
                    for (int d = T.order - 1; d >= 0; --d) {
                        if (T.tab[d] >= 0) tl += std::min<int64_t>(T.dims[d], (CHl - 1) / P + 2);
                        P *= std::max<int64_t>(T.dims[d], 1);
                    }
                    if ((size_t)tl * 4 + bin_b + 16 <= kScatterSmemBudget && tl <= 16384) {
                        gtab = false;
                        ltab = true;
                        TTl = tl;
                    }
                }
                const size_t tab_b = gtab ? 0 : (size_t)TTl * 4;
                const int cls = T.order <= 2 ? 0 : (T.order <= 4 ? 1 : (T.order <= 6 ? 2 : 3));
                static const int kClassOrder[M1Plan::kOrderClasses] = {2, 4, 6, TNSK_MAX_ORDER};
                // FP32 sketches with privatised bins: the fixed-point kernel, 4-byte integer
                // bins plus an FP32 accumulator when an item spans more than one batch
                // the fixed-point kernel's four-entry loads: FP32 data, 16-byte aligned, last
                // dim a multiple of 4 (so are the chunk bounds)
                const bool vec4 = T.dtype == TNSK_F32 && T.order >= 1 && (T.dims[T.order - 1] & 3) == 0 &&
                                  ((uintptr_t)T.data & 15) == 0;
                // the item sizes: the default chunk, then the schedule's multiple of it for
                // the tensor's scatter list (kept only where the bins still fit)
                int list = 0, nrep = 1;
                int64_t CH = 8192;
                size_t bin_p = 0;
                bool priv = false;
                for (int pass = 0; pass < 2; ++pass) {
                    int scale = 1;
                    if (pass == 1 && sched && !gtab && !ltab)
                        scale = std::max(1, std::min(64, (int)sched->chunk_scale[list]));
                    if (pass == 1 && scale == 1) break;
                    const int64_t CHp = std::max<int64_t>(8192, 32 * T.O * m) * scale;
                    // FP32 tensors with a short contracted last mode whose entries cannot be
                    // read four at a time take the fiber kernel (m1_scatter_fiber.cu): its
                    // batches are whole fibers, so the bins allow for either kernel's batch
                    const int Ld = T.dims[T.order - 1];
                    const bool fib_shape = !fp64 && !vec4 && !gtab && T.dtype == TNSK_F32 && T.order >= 2 && Ld >= 2 &&
                                           Ld <= 16;
                    const int64_t batch = fib_shape ? std::min<int64_t>(m1_fx_batch(kClassOrder[cls]), m1_fiber_batch(Ld))
                                                    : m1_fx_batch(kClassOrder[cls]);
                    const bool fx_multi = std::min<int64_t>(T.numel, CHp) > batch;
                    const size_t bin_fx = (size_t)T.O * m * 4 * (fx_multi ? 2 : 1);
                    // (bins that fit only as FP32 words keep the atomic kernel)
                    const bool fx = !fp64 && tab_b + bin_fx + 16 <= kScatterSmemBudget;
                    const size_t bp = fx ? bin_fx : bin_b;
                    const int64_t nrep_priv = (int64_t)(kScatterSmemBudget / (tab_b + bp + 16));
                    const bool pv = nrep_priv >= 1 && T.numel * 4 >= T.O * m;
                    const int kind = (fx && pv) ? (vec4 ? 1 : (fib_shape ? 3 : 2)) : 0;
                    const int l = cls + M1Plan::kOrderClasses * kind;
                    if (pass == 1 && l != list) break;  // the larger chunk would change the kernel
                    list = l;
                    priv = pv;
                    bin_p = bp;
                    const int cap = sched && sched->rep_cap[l] > 0 ? (int)sched->rep_cap[l] : (pv ? 32 : 16);
                    if (pv)
                        nrep = (int)std::min<int64_t>({(int64_t)R, nrep_priv, std::min(cap, 32)});
                    else
                        nrep = (int)std::min<int64_t>(
                            {(int64_t)R, std::max<int64_t>(1, (int64_t)(kScatterSmemBudget / (tab_b + 16))),
                             std::min(cap, 16)});
                    // chunks: privatised bins are flushed once per chunk, so a chunk has at
                    // least 32x as many entries as bins (a few percent of flush per update)
                    CH = pv ? CHp : (gtab ? 65536 : 8192) * scale;
                    if (kind == 3) CH = CHp / Ld * Ld;  // whole fibers per item
                }
                size_t sm = ((size_t)nrep * tab_b + 15) / 16 * 16 + (priv ? (size_t)nrep * bin_p : 0);
                P.m1.class_smem[list] = std::max(P.m1.class_smem[list], sm);
                for (int r0 = 0; r0 < R; r0 += nrep)
                    for (int64_t b0 = 0; b0 < T.numel; b0 += CH) {
                        M1Work w{};
                        w.begin = b0;
                        w.end = std::min(T.numel, b0 + CH);
                        w.tensor = nb.t0 + k;
                        w.rep0 = r0;
                        w.nrep = std::min(nrep, R - r0);
                        w.priv = priv ? ((w.begin == 0 && w.end == T.numel) ? 2 : 1) : 0;
                        w.gtab = gtab ? 1 : 0;
                        w.ltab = ltab ? 1 : 0;
                        m1w_cls[list].push_back(w);
                    }
            }
            const bool large = I.log2m > max_log2m_for(fp64);
            if (large && (nb.n_ot > 0 || I.O > 1)) {
                err = "method 1 above m = 2^14 (FP32) / 2^13 (FP64) takes networks without open legs only";
                return TNSK_ERR_UNSUPPORTED;
            }
            if (!sketch_only && I.O > 0 && large) {
                // packed transforms (M = m/2 complex values per sketch) through a global
                // scratch: pass 1 per (rep, sketch), pass 2 and the product per (rep,
                // pair of rows {k1, N1 - k1}, k1 <= N1/2), G sketches of a rep at a time
                nb.lspec_off = lspec_n;
                lspec_n += (int64_t)R * I.p * (m / 2);
                const int LM = I.log2m - 1, N1 = 1 << (LM / 2);
                const int G = m1_large_rows_group(I.log2m, I.p, fp64);
                P.m1.lrows_smem = std::max(P.m1.lrows_smem, m1_large_rows_smem(I.log2m, G, fp64));
                for (int r = 0; r < R; ++r) {
                    for (int k = 0; k < I.p; ++k) lfft.push_back(make_int4((int)m1n.size(), r, k, 0));
                    for (int k1 = 0; k1 <= N1 / 2; ++k1) lprod.push_back(make_int4((int)m1n.size(), r, k1, G));
                }
            } else if (!sketch_only && I.O == 1 && nb.n_ot == 0 && I.log2m >= 11) {
                // closed networks at 2^11 <= m <= 2^14 (2^13 FP64): one CTA per sketch for
                // the transforms, half spectra [R][p][m/2 + 1] through a global scratch
                const int64_t K = (m >> 1) + 1;
                nb.lspec_off = lspec_n;
                lspec_n += (int64_t)R * I.p * K;
                mid_max_log2m = std::max(mid_max_log2m, I.log2m);
                for (int r = 0; r < R; ++r) {
                    for (int k = 0; k < I.p; ++k) mfft.push_back(make_int4((int)m1n.size(), r, k, 0));
                    for (int64_t j0 = 0; j0 < K; j0 += 4096)
                        mprod.push_back(make_int4((int)m1n.size(), r, (int)j0, (int)std::min<int64_t>(4096, K - j0)));
                }
            } else if (!sketch_only && I.O > 0) {
                // FP32, 2^6 <= m <= 2^10: the warp-per-item spectrum kernel
                const bool warp_path = !fp64 && I.log2m >= 6 && I.log2m <= 10;
                std::vector<int2>& dst = warp_path ? m1warp[I.log2m - 6] : m1items;
                // the block kernel's shared memory is sized by the largest m it runs
                if (!warp_path) max_log2m1 = std::max(max_log2m1, I.log2m);
                for (int r = 0; r < R; ++r) dst.push_back(make_int2((int)m1n.size(), r));
            }
            if (sketch_only) P.sketch_user_bytes = (size_t)R * xacc * acc;
            xs_n += sketch_only ? 0 : (int64_t)R * xacc;
            xs_n = (xs_n + 3) & ~(int64_t)3;  // every network's sketches start 16-byte aligned
            spec_n += (int64_t)R * sacc;
            sexp_n += (int64_t)R * eacc;
            for (int64_t o = 0; o < I.O; ++o) {
                CombineItem c{};
                c.y_off = yrep_n;
                c.O = I.O;
                c.o = o;
                c.R = R;
                c.groups = pr.groups;
                c.out = nb.out;
                c.per_rep = nb.per_rep;
                c.ps = I.O;
                comb.push_back(c);
            }
            yrep_n += (int64_t)R * I.O;
            if (m1n.empty()) P.m1_reps = R;
            m1n.push_back(nb);
            continue;
        }
        // ---------------- method 2 ----------------
        M2Net nb{};
        nb.m = m;
        nb.log2m = I.log2m;
        nb.R = R;
        nb.tab_off = tab_words;
        // reps per row-scatter CTA: at most 4 (enough CTAs to fill the GPU), bins of up
        // to 48 KiB in shared memory
        const int scatter_reps = (int)std::max<int64_t>(1, std::min<int64_t>(4, (48 * 1024) / (m * 4)));
        P.m2.scatter_smem = std::max(P.m2.scatter_smem, (size_t)scatter_reps * (size_t)m * sizeof(float));
        nb.y_off = yrep_n;
        max_log2m2 = std::max(max_log2m2, I.log2m);
        const int net_id = (int)m2n.size();
        const size_t node0 = m2nodes.size();
        std::vector<int> qt(I.p, 0);
        int64_t Lrep = I.L;
        std::vector<int64_t> pad_tab(I.p), t_tab(I.p);
        for (int k = 0; k < I.p; ++k) {
            int c = (int)I.child[k].size();
            while (qt[k] < c) qt[k] = qt[k] ? qt[k] * 2 : 1;
            pad_tab[k] = Lrep;
            Lrep += qt[k];
        }
        for (int k = 0; k < I.p; ++k) {
            t_tab[k] = Lrep;
            if (qt[k] >= 2) Lrep += 2 * (int64_t)(qt[k] - 1) * m;
        }
        nb.Lrep = Lrep;
        // tables: C_{k,l} per edge, padding slots, T_{l,j} (Alg. 2 "independent recursive sketch")
        for (int e = 0; e < I.t; ++e) {
            TabReq q{};
            q.seed = pr.seed;
            q.rep_base = pr.rep0;
            q.tid = tid_m2_edge(e);
            q.n = I.eoff[e + 1] - I.eoff[e];
            q.out_off = tab_words + I.eoff[e];
            q.rep_stride = Lrep;
            q.R = R;
            q.mask = mask;
            if (q.n > 0) reqs.push_back(q);
        }
        for (int k = 0; k < I.p; ++k) {
            int c = (int)I.child[k].size();
            for (int j = c; j < qt[k]; ++j) {
                TabReq q{};
                q.seed = pr.seed;
                q.rep_base = pr.rep0;
                q.tid = tid_m2_pad(k, j);
                q.n = 1;
                q.out_off = tab_words + pad_tab[k] + j;
                q.rep_stride = Lrep;
                q.R = R;
                q.mask = mask;
                reqs.push_back(q);
            }
            for (int l = qt[k]; l >= 2; l >>= 1)
                for (int j = 0; j < l / 2; ++j)
                    for (int s = 0; s < 2; ++s) {
                        TabReq q{};
                        q.seed = pr.seed;
                        q.rep_base = pr.rep0;
                        q.tid = tid_m2_ts(k, ilog2(l), j, s);
                        q.n = m;
                        q.out_off = tab_words + t_tab[k] + ts_offset(qt[k], l, j, s, m);
                        q.rep_stride = Lrep;
                        q.R = R;
                        q.mask = mask;
                        reqs.push_back(q);
                    }
        }
        tab_words += (int64_t)R * Lrep;
        // nodes
        auto up16 = [](int64_t v) { return (v + 15) & ~(int64_t)15; };
        std::vector<int64_t> xo(I.p, -1);
        for (int k = 0; k < I.p; ++k) {
            if (k == I.root) continue;
            xo[k] = ws_x;
            ws_x = up16(ws_x + (int64_t)R * m);
        }
        for (int k = 0; k < I.p; ++k) {
            const tnsk_tensor& X = N.X[k];
            M2Node nd{};
            nd.data = X.data;
            nd.numel = I.numel[k];
            nd.dtype = X.dtype;
            nd.order = X.order;
            nd.net = net_id;
            nd.is_root = k == I.root;
            nd.pmode = I.parent_mode[k];
            for (int d = 0; d < X.order; ++d) nd.dims[d] = (int32_t)I.dims[I.mode_off[k] + d];
            if (nd.is_root) {
                nd.A = 1;
                nd.npar = 1;
                nd.Bc = nd.numel;
            } else {
                nd.A = 1;
                nd.Bc = 1;
                for (int d = 0; d < nd.pmode; ++d) nd.A *= nd.dims[d];
                for (int d = nd.pmode + 1; d < X.order; ++d) nd.Bc *= nd.dims[d];
                nd.npar = nd.dims[nd.pmode];
            }
            nd.cols = nd.A * nd.Bc;
            if (nd.cols >= ((int64_t)1 << 32)) {
                if (nd.A > 1) {
                    err = "tensor " + std::to_string(k) + ": 2^32 or more columns with the parent mode not first";
                    return TNSK_ERR_UNSUPPORTED;
                }
                P.m2.idx32 = false;
            }
            nd.ptab = nd.is_root ? -1 : I.eoff[I.parent_edge[k]];
            nd.c = (int)I.child[k].size();
            if (I.rung[k]) {
                // grouped tensor: generated inside the sketch product, so it must be an inner
                // node (leaves and the root read their entries directly)
                const tnsk_rung& g = *I.rung[k];
                if (nd.is_root || nd.c == 0 || nd.order != 2) {
                    err = "tensor " + std::to_string(k) + ": a rung tensor must be an inner node of the rooted tree";
                    return TNSK_ERR_UNSUPPORTED;
                }
                const bool first = nd.pmode == 0;  // rows (i, j), columns (k, l); else transposed
                nd.rA = (const float*)g.A;
                nd.rB = (const float*)g.B;
                nd.rs = (int32_t)g.s;
                nd.rn_i1 = (int32_t)(first ? g.a : g.c);
                nd.rn_i2 = (int32_t)(first ? g.b : g.d);
                nd.rn_j1 = (int32_t)(first ? g.c : g.a);
                nd.rn_j2 = (int32_t)(first ? g.d : g.b);
                // A(i, s, k) at i s c + s c + k; B(j, s, l) at j s d + s d + l
                nd.r_as = (int32_t)g.c;
                nd.r_bs = (int32_t)g.d;
                nd.r_ai = (int32_t)(first ? g.s * g.c : 1);
                nd.r_aj = (int32_t)(first ? 1 : g.s * g.c);
                nd.r_bi = (int32_t)(first ? g.s * g.d : 1);
                nd.r_bj = (int32_t)(first ? 1 : g.s * g.d);
                const int64_t b_bytes = (int64_t)nd.rn_i2 * (g.s * nd.rn_j2 + 4) * 4;
                const bool tc_ok = nd.rn_j2 % 32 == 0 && b_bytes <= 60 * 1024 && tma;
                // all four factor dims 32 and s <= 8: the factored product on the tensor
                // cores (m2_rung_tc.cu), which neither forms X's entries nor reads them
                const bool tc_fact = tma && nd.rn_i1 == 32 && nd.rn_i2 == 32 && nd.rn_j1 == 32 &&
                                     nd.rn_j2 == 32 && g.s >= 1 && g.s <= 8;
                nd.r_fact = tc_fact ? 2 : (!tc_ok && rung_small(g) ? 1 : 0);
                if (nd.r_fact == 1) {
                    P.m2.rungf_smem = std::max(P.m2.rungf_smem, m2_rung_fact_smem((int)g.s));
                } else if (!tc_ok && !tc_fact) {
                    err = "tensor " + std::to_string(k) +
                          ": rung tensor needs factor dims <= 32, or its column fast index a multiple of 32 and the "
                          "B factor within 60 KiB";
                    return TNSK_ERR_UNSUPPORTED;
                }
                // A rows of a 128-row tile: at most 127 / n_i2 + 2 values of i1, staged when
                // they fit 16 KiB
                const int64_t i1_max = std::min<int64_t>(nd.rn_i1, 127 / nd.rn_i2 + 2);
                const int64_t a_bytes = i1_max * g.s * nd.rn_j1 * 4;
                nd.r_astage = a_bytes <= 16 * 1024 ? 1 : 0;
                if (!nd.r_fact)
                    P.m2.rung_smem = std::max(P.m2.rung_smem,
                                              m2_gemm_rung_smem((size_t)(b_bytes + (nd.r_astage ? a_bytes : 0))));
            }
            nd.qt = qt[k];
            P.m2.max_qt = std::max(P.m2.max_qt, nd.qt);
            P.m2.max_order = std::max(P.m2.max_order, nd.order);
            for (int j = 0; j < nd.c; ++j) {
                nd.cmode[j] = I.child_mode[k][j];
                nd.ctab[j] = I.eoff[I.child_edge[k][j]];
            }
            nd.pad_tab = pad_tab[k];
            nd.t_tab = t_tab[k];
            nd.tm_x = -1;
            nd.tm_v = -1;
            nd.rc_off = -1;
            M2Fix fx{};
            fx.node = m2nodes.size();
            fx.x = xo[k];
            fx.r = -1;
            fx.v = -1;
            fx.c = -1;
            if (nd.r_fact == 2) {
                fx.c = ws_c;
                ws_c = up16(ws_c + 4 * (int64_t)nd.rs * 1024);
            }
            fx.src_kind = 0;
            for (int j = 0; j < nd.c; ++j) fx.child_x[j] = xo[I.child[k][j]];
            if (nd.qt >= 2) {
                fx.r = ws_r;
                ws_r = up16(ws_r + (int64_t)R * (nd.qt - 1) * m);
                fx.src = fx.r + (int64_t)(nd.qt - 2) * m;
                fx.src_kind = 1;
                nd.src_stride = (int64_t)(nd.qt - 1) * m;
            } else if (nd.qt == 1) {
                fx.src = xo[I.child[k][0]];
                fx.src_kind = 2;
                nd.src_stride = m;
            }
            if (nd.c >= 1) {
                fx.v = ws_v;
                const int64_t parts = (!fp64 && !nd.is_root) ? 2 : 1;  // TF32 hi / lo for the tensor cores
                ws_v = up16(ws_v + parts * nd.cols * (int64_t)R);
            }
            fx.w = -1;
            if (!fp64 && nd.c >= 1 && !nd.is_root) {  // tensor-core product W^T
                fx.w = ws_w;
                ws_w = up16(ws_w + nd.npar * (int64_t)R);
            }
            fixes.push_back(fx);
            m2nodes.push_back(nd);
            // work items at this node's height
            const int h = I.height[k];
            const int node_idx = (int)(node0 + k);
            if (nd.c == 0 && !nd.is_root) {  // chunks of 2048 entries x blocks of 8 reps
                for (int64_t b0 = 0; b0 < nd.numel; b0 += 2048)
                    for (int r0 = 0; r0 < R; r0 += 8) {
                        M2Item it{node_idx, r0, std::min(8, R - r0), 0, b0, std::min(nd.numel, b0 + 2048)};
                        pend.push_back({h, M2_LEAF, it});
                    }
            }
            if (nd.qt >= 2)
                for (int r = 0; r < R; ++r) pend.push_back({h, M2_COMPOSE, M2Item{node_idx, r, 0, 0, 0, 0}});
            if (nd.c >= 1) {
                // Items of about 1-4 K outputs (enough CTAs in flight to hide the gathers'
                // latency). Where a rep's T tables (qt >= 2) and child sketch fit 48 KiB and
                // there are enough columns to amortise the copy: staged form (pad_ = 1), a
                // few reps x 512 columns with the reps' T tables and child sketches in
                // shared memory (the gathers from the child sketch are random: from L2 each
                // would move a 32-byte sector for 4 bytes). Otherwise 128 columns x 8 reps,
                // every lookup from L2.
                const int64_t tw = nd.qt >= 2 ? 2 * (int64_t)(nd.qt - 1) * m : 0;
                const int64_t per_rep = tw * 4 + m * (fp64 ? 8 : 4) + 16;
                const int64_t budget = 48 * 1024;
                if (per_rep <= budget && nd.cols >= std::max<int64_t>(256, m / 4)) {
                    const int G = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)R, budget / per_rep, nd.qt >= 2 ? 4 : 2}));
                    const int64_t cb = nd.qt >= 2 ? 512 : 2048;
                    for (int r0 = 0; r0 < R; r0 += G)
                        for (int64_t b0 = 0; b0 < nd.cols; b0 += cb) {
                            const int g = std::min(G, R - r0);
                            M2Item it{node_idx, r0, g, 1, b0, std::min(nd.cols, b0 + cb)};
                            pend.push_back({h, M2_VBUILD, it});
                            const size_t bytes =
                                (((size_t)g * tw * 4 + 15) & ~(size_t)15) + (size_t)g * m * (fp64 ? 8 : 4);
                            P.m2.vbuild_smem = std::max(P.m2.vbuild_smem, bytes);
                        }
                } else {
                    for (int r0 = 0; r0 < R; r0 += 8)
                        for (int64_t b0 = 0; b0 < nd.cols; b0 += 128) {
                            M2Item it{node_idx, r0, std::min(8, R - r0), 0, b0, std::min(nd.cols, b0 + 128)};
                            pend.push_back({h, M2_VBUILD, it});
                        }
                }
            }
            if (!fp64 && nd.c >= 1 && !nd.is_root) {
                // count sketch of W's rows into x_k, after the tensor-core product
                for (int r0 = 0; r0 < R; r0 += scatter_reps) {
                    M2Item it{node_idx, r0, std::min(scatter_reps, R - r0), 0, 0, 0};
                    pend.push_back({h, M2_WSCATTER, it});
                }
            }
            if (nd.c >= 1 && !nd.is_root && nd.numel > 0) {
                // row tiles: 128 rows for the tensor-core kernels (FP32), 64 for the FP64 one;
                // the split of K (tensor-core kernels) is chosen once all tiles are known
                const int64_t tile = fp64 ? 64 : 128;
                const bool rung = I.rung[k] != nullptr;
                if (rung && m2nodes.back().r_fact == 1) {  // blocks of 4 reps, no tiles or K split
                    for (int r0 = 0; r0 < R; r0 += 4)
                        pend.push_back({h, M2_GEMM_RUNGF, M2Item{node_idx, r0, std::min(4, R - r0), 0, 0, 0}});
                } else if (rung && m2nodes.back().r_fact == 2) {
                    // blocks of 4 reps for the persistent kernel; V^T viewed as [R 32][32] in
                    // boxes of 128 rows (hi, lo); the factors prepared once at height 0
                    m2nodes.back().tm_v = (int32_t)P.m2.tmap_jobs.size();
                    P.m2.tmap_jobs.push_back({(int)(m2nodes.size() - 1), 7});
                    P.m2.tmap_jobs.push_back({(int)(m2nodes.size() - 1), 8});
                    pend.push_back({0, M2_RUNG_PREP, M2Item{node_idx, 0, 0, 0, 0, 0}});
                    for (int r0 = 0; r0 < R; r0 += 4)
                        pend.push_back({h, M2_GEMM_RUNGT, M2Item{node_idx, r0, std::min(4, R - r0), 0, 0, 0}});
                } else {
                    const bool stream = !rung && !fp64 && tma && nd.dtype == TNSK_F32 && nd.A == 1 &&
                                        (nd.cols % 4) == 0 && ((uintptr_t)nd.data % 16) == 0 &&
                                        nd.npar < ((int64_t)1 << 31) && nd.cols < ((int64_t)1 << 31);
                    // TNSK_PREC_BF16: BF16 tensors in the same layout on the kind::f16 kernel
                    const bool bf16k = !rung && !fp64 && tma && pr.prec == TNSK_PREC_BF16 &&
                                       nd.dtype == TNSK_BF16 && nd.A == 1 && (nd.cols % 8) == 0 &&
                                       ((uintptr_t)nd.data % 16) == 0 && nd.npar < ((int64_t)1 << 31) &&
                                       nd.cols < ((int64_t)1 << 31);
                    if (bf16k) {
                        M2Node& bn = m2nodes.back();
                        bn.vbf16 = 1;
                        bn.tm_x = (int32_t)P.m2.tmap_jobs.size();
                        P.m2.tmap_jobs.push_back({(int)(m2nodes.size() - 1), 3});
                        bn.tm_v = (int32_t)P.m2.tmap_jobs.size();  // parts at tm_v, tm_v + 1, tm_v + 2
                        for (int part = 0; part < 3; ++part)
                            P.m2.tmap_jobs.push_back({(int)(m2nodes.size() - 1), 4 + part});
                    }
                    if (rung) {  // V^T hi / lo maps only: X is generated
                        m2nodes.back().tm_v = (int32_t)P.m2.tmap_jobs.size();
                        P.m2.tmap_jobs.push_back({(int)(m2nodes.size() - 1), 1});
                        P.m2.tmap_jobs.push_back({(int)(m2nodes.size() - 1), 2});
                    }
                    if (stream && !bf16k) {
                        m2nodes.back().tm_x = (int32_t)P.m2.tmap_jobs.size();
                        P.m2.tmap_jobs.push_back({(int)(m2nodes.size() - 1), 0});
                        m2nodes.back().tm_v = (int32_t)P.m2.tmap_jobs.size();  // hi, then lo at tm_v + 1
                        P.m2.tmap_jobs.push_back({(int)(m2nodes.size() - 1), 1});
                        P.m2.tmap_jobs.push_back({(int)(m2nodes.size() - 1), 2});
                    }
                    for (int64_t rt = 0; rt * tile < nd.npar; ++rt)
                        for (int64_t ct = 0; ct * 64 < R; ++ct)
                            pend.push_back({h, rung ? M2_GEMM_RUNG
                                                    : (bf16k ? M2_GEMM_BF16 : (stream ? M2_GEMM_STREAM : M2_GEMM)),
                                            M2Item{node_idx, (int)rt, (int)ct, 0, 1, 0}});
                }
            }
            if (nd.is_root)  // chunks of 4096 columns x blocks of 8 reps (one warp each)
                for (int64_t b0 = 0; b0 < std::max<int64_t>(nd.cols, 1); b0 += 4096)
                    for (int r0 = 0; r0 < R; r0 += 8) {
                        M2Item it{node_idx, r0, std::min(8, R - r0), 0, b0, std::min(nd.cols, b0 + 4096)};
                        pend.push_back({h, M2_ROOT, it});
                    }
        }
        P.m2.max_height = std::max(P.m2.max_height, I.max_height);
        CombineItem c{};
        c.y_off = yrep_n;
        c.O = 1;
        c.o = 0;
        c.R = R;
        c.groups = pr.groups;
        c.out = outs ? outs[b] : nullptr;
        c.per_rep = per_reps ? per_reps[b] : nullptr;
        c.ps = rep_stride && rep_stride[b] > 0 ? rep_stride[b] : 1;
        comb.push_back(c);
        yrep_n += R;
        m2n.push_back(nb);
    }

    // ---- method-2 workspace offsets: ws = [x | r | V] (elements of the accumulator type)
    for (const M2Fix& fx : fixes) {
        M2Node& nd = m2nodes[fx.node];
        nd.x_off = fx.x;
        nd.w_off = fx.w >= 0 ? ws_x + fx.w : -1;
        nd.r_off = fx.r >= 0 ? ws_x + ws_w + fx.r : -1;
        nd.v_off = fx.v >= 0 ? ws_x + ws_w + ws_r + fx.v : -1;
        nd.rc_off = fx.c >= 0 ? ws_x + ws_w + ws_r + ws_v + fx.c : -1;
        nd.src_off = fx.src_kind == 1 ? ws_x + ws_w + fx.src : (fx.src_kind == 2 ? fx.src : -1);
        for (int j = 0; j < nd.c; ++j) nd.child_x[j] = fx.child_x[j];
    }
    // ---- split K of the tensor-core GEMM tiles: both kernels run 2 CTAs per SM, so a
    // height's tiles x splits CTAs run in waves of 304; pick the split that minimises
    // waves x (chunks per split + a fixed cost of about 6 chunks per CTA), with at least
    // 4 chunks of 32 columns per split
    if (!fp64 && !pend.empty()) {
        std::vector<int64_t> tiles(P.m2.max_height + 1, 0);
        for (const PendingItem& q : pend)
            if (q.kind == M2_GEMM || q.kind == M2_GEMM_STREAM || q.kind == M2_GEMM_RUNG || q.kind == M2_GEMM_BF16)
                tiles[q.h]++;
        std::vector<PendingItem> out;
        out.reserve(pend.size());
        for (const PendingItem& q : pend) {
            if (q.kind != M2_GEMM && q.kind != M2_GEMM_STREAM && q.kind != M2_GEMM_RUNG && q.kind != M2_GEMM_BF16) {
                out.push_back(q);
                continue;
            }
            const int64_t kc = q.kind == M2_GEMM_BF16 ? 64 : 32;  // columns per chunk of the kernel
            const int64_t chunks = (m2nodes[q.it.node].cols + kc - 1) / kc;
            const int64_t slots = 2 * 152, fixed = 6;
            int64_t split = 1, best = -1;
            for (int64_t sp = 1; sp <= std::max<int64_t>(1, std::min<int64_t>(chunks / 4, 64)); ++sp) {
                const int64_t waves = (tiles[q.h] * sp + slots - 1) / slots;
                const int64_t cost = waves * ((chunks + sp - 1) / sp + fixed);
                if (best < 0 || cost < best) best = cost, split = sp;
            }
            for (int64_t sidx = 0; sidx < split; ++sidx) {
                PendingItem z = q;
                z.it.begin = split;  // number of K splits
                z.it.pad_ = (int)sidx;
                out.push_back(z);
            }
        }
        pend.swap(out);
    }
    // ---- method-2 item order: by height, then kind
    std::vector<M2Item>& m2items = L.m2items;
    if (!m2n.empty()) {
        const int H = P.m2.max_height + 1;
        P.m2.first.assign(H * M2_NKINDS, 0);
        P.m2.count.assign(H * M2_NKINDS, 0);
        std::stable_sort(pend.begin(), pend.end(), [](const PendingItem& a, const PendingItem& b) {
            return a.h != b.h ? a.h < b.h : a.kind < b.kind;
        });
        for (size_t i = 0; i < pend.size(); ++i) {
            int slot = pend[i].h * M2_NKINDS + pend[i].kind;
            if (P.m2.count[slot] == 0) P.m2.first[slot] = (int)i;
            P.m2.count[slot]++;
            m2items.push_back(pend[i].it);
        }
    }
    P.m2.n_nets = (int)m2n.size();
    P.m2.max_log2m = max_log2m2;

    // ---- table request prefix offsets
    int64_t crow = 0;
    for (TabReq& q : reqs) {
        q.crow = crow;
        crow += q.R;
    }
    P.n_reqs = (int)reqs.size();
    P.n_table_rows = crow;

    // ---- row-sorted sketches: the concatenation of every entry's (strip, sorted row)
    // positions split into one equal contiguous part per CTA slot (m1_rowsort_slots)
    if (!rsorts.empty()) {
        std::vector<int64_t> start(rsorts.size() + 1, 0);
        for (size_t i = 0; i < rsorts.size(); ++i) {
            const M1Tensor& T = m1t[rsorts[i].tensor];
            start[i + 1] = start[i] + (int64_t)rsorts[i].strips * T.dims[0];
        }
        const int64_t total = start.back();
        const int64_t G = std::max<int64_t>(1, std::min<int64_t>(m1_rowsort_slots(), total / 64));
        size_t e = 0;
        for (int64_t g = 0; g < G; ++g) {
            const int64_t a = total * g / G, b = total * (g + 1) / G;
            if (b <= a) continue;
            while (start[e + 1] <= a) ++e;
            const int64_t n0 = m1t[rsorts[e].tensor].dims[0];
            const int64_t off = a - start[e];
            ritems.push_back(M1RowItem{(int)e, (int)(off / n0), (int)(off % n0), 0, b - a});
        }
        int64_t most_n0 = 0;
        for (const M1RowSort& r : rsorts) most_n0 = std::max<int64_t>(most_n0, m1t[r.tensor].dims[0]);
        P.m1.rs_max_rows = (int)most_n0;
    }

    // ---- stage descriptors
    std::vector<unsigned char>& H = P.host_desc;
    for (int c = 0; c < M1Plan::kScatterLists; ++c) {
        P.m1.work_first[c] = (int)m1w.size();
        P.m1.work_count[c] = (int)m1w_cls[c].size();
        m1w.insert(m1w.end(), m1w_cls[c].begin(), m1w_cls[c].end());
    }
    // the per-rep magnitude sums of method-1 networks follow all per-rep estimates
    for (M1Net& nb : m1n) nb.yabs_off = nb.y_off + yrep_n;
    {
        // one allocation for the staged block (a recycled one where the thread has it)
        size_t total = 0;
        auto add = [&](size_t bytes) { total = ((total + 255) & ~(size_t)255) + bytes; };
        add(reqs.size() * sizeof(TabReq));
        add(m1t.size() * sizeof(M1Tensor));
        add(m1n.size() * sizeof(M1Net));
        add(m1w.size() * sizeof(M1Work));
        size_t n_items = m1items.size();
        for (int sl = 0; sl < M1Plan::kWarpSlots; ++sl) n_items += m1warp[sl].size();
        add(opens.size() * sizeof(OpenMode));
        add(n_items * sizeof(int2));
        add(comb.size() * sizeof(CombineItem));
        for (size_t n : {lfft.size(), lprod.size()}) add(n * sizeof(int4));
        add(diags.size() * sizeof(M1Diag));
        for (size_t n : {mfft.size(), mprod.size()}) add(n * sizeof(int4));
        add(rsorts.size() * sizeof(M1RowSort));
        add(ritems.size() * sizeof(M1RowItem));
        add(m2nodes.size() * sizeof(M2Node));
        add(m2n.size() * sizeof(M2Net));
        add(m2items.size() * sizeof(M2Item));
        add(P.m2.tmap_jobs.size() * 128);
        take_desc_buffer(H);
        H.reserve(total);
    }
    size_t o_reqs = stage(H, reqs), o_m1t = stage(H, m1t), o_m1n = stage(H, m1n), o_m1w = stage(H, m1w);
    const int n_block_items = (int)m1items.size();
    for (int sl = 0; sl < M1Plan::kWarpSlots; ++sl) {
        P.m1.warp_first[sl] = (int)m1items.size();
        P.m1.warp_count[sl] = (int)m1warp[sl].size();
        m1items.insert(m1items.end(), m1warp[sl].begin(), m1warp[sl].end());
    }
    size_t o_open = stage(H, opens), o_items = stage(H, m1items), o_comb = stage(H, comb);
    size_t o_lfft = stage(H, lfft), o_lprod = stage(H, lprod), o_diag = stage(H, diags);
    size_t o_mfft = stage(H, mfft), o_mprod = stage(H, mprod);
    size_t o_rs = stage(H, rsorts), o_ritems = stage(H, ritems);
    size_t o_m2nodes = stage(H, m2nodes), o_m2n = stage(H, m2n), o_m2items = stage(H, m2items);
    std::vector<unsigned char> tmap_space(P.m2.tmap_jobs.size() * 128, 0);
    size_t o_tmaps = stage(H, tmap_space);
    P.desc_off = P.arena.take(H.size());
    P.reqs_off = P.desc_off + o_reqs;
    P.m1.tens_off = P.desc_off + o_m1t;
    P.m1.nets_off = P.desc_off + o_m1n;
    P.m1.work_off = P.desc_off + o_m1w;
    P.m1.opens_off = P.desc_off + o_open;
    P.m1.items_off = P.desc_off + o_items;
    P.m1.lfft_off = P.desc_off + o_lfft;
    P.m1.lprod_off = P.desc_off + o_lprod;
    P.m1.n_lfft = (int)lfft.size();
    P.m1.n_lprod = (int)lprod.size();
    P.m1.mfft_off = P.desc_off + o_mfft;
    P.m1.mprod_off = P.desc_off + o_mprod;
    P.m1.n_mfft = (int)mfft.size();
    P.m1.n_mprod = (int)mprod.size();
    P.m1.mid_max_log2m = mid_max_log2m;
    P.m1.rs_off = P.desc_off + o_rs;
    P.m1.rs_items_off = P.desc_off + o_ritems;
    P.m1.n_rs = (int)rsorts.size();
    P.m1.n_rs_items = (int)ritems.size();
    P.m1.diag_off = P.desc_off + o_diag;
    P.m1.n_diag = (int)diags.size();
    for (const M1Diag& d : diags) P.m1.diag_most = std::max(P.m1.diag_most, d.n * (int64_t)m1n[d.net].R);
    P.comb_off = P.desc_off + o_comb;
    P.m2.nodes_off = P.desc_off + o_m2nodes;
    P.m2.nets_off = P.desc_off + o_m2n;
    P.m2.items_off = P.desc_off + o_m2items;
    P.m2.tmaps_off = P.desc_off + o_tmaps;
    // ---- zeroed region: per-rep estimates, method-1 sketches, method-2 x accumulators
    P.zero_off = P.arena.take(0);
    P.yrep_off = P.arena.take((size_t)2 * yrep_n * sizeof(double));  // estimates, then magnitude sums
    P.yrep_n = yrep_n;
    P.m1.xs_off = P.arena.take((size_t)xs_n * acc);
    P.m1.xs_count = xs_n;
    P.m2.ws_off = P.arena.take((size_t)(ws_x + ws_w + ws_r + ws_v + ws_c) * acc);
    P.zero_bytes = P.m2.ws_off + (size_t)(ws_x + ws_w) * acc - P.zero_off;
    // ---- the rest
    P.tabs_off = P.arena.take((size_t)tab_words * sizeof(uint32_t));
    P.m1.spec_off = P.arena.take((size_t)spec_n * 2 * acc);
    P.m1.lspec_off = P.arena.take((size_t)lspec_n * 2 * acc);
    P.m1.sexp_off = P.arena.take((size_t)sexp_n * sizeof(int));
    P.m1.rs_scratch_off = P.arena.take((size_t)rs_words * sizeof(uint32_t));
    P.m1.n_nets = (int)m1n.size();
    P.m1.n_work = (int)m1w.size();
    P.m1.n_items = n_block_items;
    P.m1.max_log2m = max_log2m1;
    P.n_comb = (int)comb.size();
    return TNSK_OK;
}

}  // namespace tnsk
