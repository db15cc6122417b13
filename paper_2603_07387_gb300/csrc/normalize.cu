// normalize.cu -- the WLOG rewrites of Sec. 4.1: copy tensors for hyperedges (WLOG 1,
// method-1 kernels) and the WLOG 2 / WLOG 3 rewrite for the acyclic method (host
// bookkeeping and the one kernel that writes the rewritten tensors).
#include <algorithm>
#include <limits>
#include <map>
#include <utility>

#include "normalize.cuh"
#include "plan.cuh"

namespace tnsk {

// One thread per output entry: decode its index over the kept modes (in their new
// order) into a source offset, then sum the traced diagonals (mixed-radix counter
// over the traced pairs; no pair: a plain gather).
__global__ void __launch_bounds__(256) normalize_kernel(const NormJob* __restrict__ jobs) {
    const NormJob& J = jobs[blockIdx.y];
    const int64_t numel = J.numel;
    const int n = J.n, nd = J.nd;
    bool empty = false;
    for (int j = 0; j < nd; ++j) empty |= J.ddim[j] == 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < numel;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t rem = i, off = 0;
        for (int j = n - 1; j >= 0; --j) {
            const int64_t q = rem / J.dim[j];
            off += (rem - q * J.dim[j]) * J.str[j];
            rem = q;
        }
        double acc = 0.0;
        if (nd == 0) {
            acc = load_as<double>(J.src, J.src_dtype, off);
        } else if (!empty) {
            int64_t c[TNSK_MAX_ORDER / 2] = {};
            for (;;) {
                acc += load_as<double>(J.src, J.src_dtype, off);
                int j = nd - 1;
                for (; j >= 0; --j) {
                    if (++c[j] < J.ddim[j]) {
                        off += J.dstr[j];
                        break;
                    }
                    off -= (J.ddim[j] - 1) * J.dstr[j];
                    c[j] = 0;
                }
                if (j < 0) break;
            }
        }
        if (J.dst_f64)
            static_cast<double*>(J.dst)[i] = acc;
        else
            static_cast<float*>(J.dst)[i] = (float)acc;
    }
}

cudaError_t launch_normalize(const NormJob* d_jobs, int n, int64_t most, cudaStream_t s) {
    if (n <= 0 || most <= 0) return cudaSuccess;
    const unsigned gx = (unsigned)std::min<int64_t>((most + 255) / 256, 4096);
    for (int first = 0; first < n; first += 65535) {
        const unsigned gy = (unsigned)std::min(65535, n - first);
        normalize_kernel<<<dim3(gx, gy), 256, 0, s>>>(d_jobs + first);
    }
    return cudaGetLastError();
}

namespace {

// True when an acyclic network needs the WLOG 2 / 3 rewrite (a contraction inside one
// tensor, or two between one pair); false when it needs none or fails the basic
// checks (left to planning). Fills the mode owners, dims and per-tensor mode offsets.
bool needs_rewrite(const tnsk_network& N, std::vector<int>& owner, std::vector<int64_t>& dimg,
                   std::vector<int>& moff) {
    if (N.p < 1 || !N.X || N.t < 0 || (N.t > 0 && !N.edges) || N.n_open != 0) return false;
    moff.assign(N.p + 1, 0);
    owner.clear();
    dimg.clear();
    for (int k = 0; k < N.p; ++k) {
        const tnsk_tensor& X = N.X[k];
        if (X.order < 0 || X.order > TNSK_MAX_ORDER || (X.order > 0 && !X.dims)) return false;
        int64_t numel = 1;
        for (int d = 0; d < X.order; ++d) {
            if (X.dims[d] < 0 || X.dims[d] > std::numeric_limits<int32_t>::max()) return false;
            owner.push_back(k);
            dimg.push_back(X.dims[d]);
            numel *= X.dims[d] > 0 ? 1 : 0;
        }
        if (!X.data && !X.rung && numel != 0) return false;
        moff[k + 1] = moff[k] + X.order;
    }
    const int q = moff[N.p];
    std::vector<char> used(q, 0);
    std::map<std::pair<int, int>, int> cnt;
    bool need = false;
    for (int e = 0; e < N.t; ++e) {
        const int u = N.edges[2 * e], v = N.edges[2 * e + 1];
        if (u < 0 || v < 0 || u >= q || v >= q || u == v || used[u] || used[v] || dimg[u] != dimg[v]) return false;
        used[u] = used[v] = 1;
        const int a = owner[u], b = owner[v];
        if (a == b || ++cnt[{std::min(a, b), std::max(a, b)}] >= 2) need = true;
    }
    return need;
}

// WLOG 1: copy tensors for the classes of three or more modes. Leaves `nn` and
// `diag` empty when the network needs none or fails the basic checks.
tnsk_status copy_tensors(const tnsk_network& N, int b, NormNet& nn, std::vector<char>& diag, std::string& why) {
    if (N.p < 1 || !N.X || N.t < 0 || (N.t > 0 && !N.edges)) return TNSK_OK;
    std::vector<int64_t> dimg;
    for (int k = 0; k < N.p; ++k) {
        const tnsk_tensor& X = N.X[k];
        if (X.order < 0 || X.order > TNSK_MAX_ORDER || (X.order > 0 && !X.dims)) return TNSK_OK;
        for (int d = 0; d < X.order; ++d) dimg.push_back(X.dims[d]);
    }
    const int q = (int)dimg.size();
    std::vector<int> uses(q, 0), parent(q);
    for (int g = 0; g < q; ++g) parent[g] = g;
    auto find = [&](int a) {
        while (parent[a] != a) a = parent[a] = parent[parent[a]];
        return a;
    };
    bool hyper = false;
    for (int e = 0; e < N.t; ++e) {
        const int u = N.edges[2 * e], v = N.edges[2 * e + 1];
        if (u < 0 || v < 0 || u >= q || v >= q || u == v || dimg[u] != dimg[v]) return TNSK_OK;
        hyper |= ++uses[u] > 1;
        hyper |= ++uses[v] > 1;
        parent[find(u)] = find(v);
    }
    if (!hyper) return TNSK_OK;
    std::map<int, std::vector<int>> members;  // class root -> its modes, ascending
    for (int g = 0; g < q; ++g)
        if (uses[g]) members[find(g)].push_back(g);
    nn.X.assign(N.X, N.X + N.p);
    nn.dims.assign(N.p, {});
    for (int e = 0; e < N.t; ++e) {  // two-mode classes: their first pair
        const int u = N.edges[2 * e], v = N.edges[2 * e + 1];
        std::vector<int>& cl = members[find(u)];
        if (cl.size() == 2 && cl[0] >= 0) {
            nn.edges.push_back(u);
            nn.edges.push_back(v);
            cl[0] = -1;  // taken
        }
    }
    std::vector<std::vector<int>> copies;
    for (auto& kv : members)
        if (kv.second.size() >= 3) copies.push_back(kv.second);
    std::sort(copies.begin(), copies.end(), [](const std::vector<int>& a, const std::vector<int>& c) {
        return a[0] < c[0];
    });
    int next = q;
    for (const std::vector<int>& cl : copies) {
        if ((int)cl.size() > TNSK_MAX_ORDER) {
            why = "network " + std::to_string(b) + ": a hyperedge joins " + std::to_string(cl.size()) +
                  " modes (its WLOG 1 copy tensor would exceed order 12)";
            return TNSK_ERR_UNSUPPORTED;
        }
        nn.dims.push_back(std::vector<int64_t>(cl.size(), dimg[cl[0]]));
        tnsk_tensor c{};
        c.order = (int32_t)cl.size();
        c.dtype = TNSK_F32;
        nn.X.push_back(c);
        for (size_t j = 0; j < cl.size(); ++j) {
            nn.edges.push_back(cl[j]);
            nn.edges.push_back(next + (int)j);
        }
        next += (int)cl.size();
    }
    for (size_t k = (size_t)N.p; k < nn.X.size(); ++k) nn.X[k].dims = nn.dims[k].data();
    nn.job.assign(nn.X.size(), -1);
    diag.assign(nn.X.size(), 0);
    for (size_t k = (size_t)N.p; k < nn.X.size(); ++k) diag[k] = 1;
    nn.net = N;
    nn.net.p = (int32_t)nn.X.size();
    nn.net.X = nn.X.data();
    nn.net.t = (int32_t)(nn.edges.size() / 2);
    nn.net.edges = nn.edges.empty() ? nullptr : nn.edges.data();
    return TNSK_OK;
}

}  // namespace

tnsk_status normalize_batch(int B, const tnsk_network* nets, const tnsk_params* params, NormBatch& nb,
                            std::string& why) {
    nb = NormBatch{};
    if (B <= 0 || !nets || !params) return TNSK_OK;
    nb.nets.resize(B);
    nb.diag.resize(B);
    nb.view.assign(nets, nets + B);
    size_t off = 0;
    std::vector<int> owner, moff;
    std::vector<int64_t> dimg;
    for (int b = 0; b < B; ++b) {
        const tnsk_network& N = nets[b];
        if (is_m1(params[b].method)) {
            tnsk_status st = copy_tensors(N, b, nb.nets[b], nb.diag[b], why);
            if (st != TNSK_OK) return st;
            if (!nb.diag[b].empty()) {
                nb.view[b] = nb.nets[b].net;
                nb.used = true;
            }
            continue;
        }
        if (params[b].method != TNSK_ACYCLIC || !needs_rewrite(N, owner, dimg, moff)) continue;
        const int p = N.p, q = moff[p], t = N.t;
        // WLOG 3 groups: the first edge of each pair of tensors joined more than once
        std::map<std::pair<int, int>, int> first, count;
        for (int e = 0; e < t; ++e) {
            const int a = owner[N.edges[2 * e]], c = owner[N.edges[2 * e + 1]];
            if (a == c) continue;
            const std::pair<int, int> key{std::min(a, c), std::max(a, c)};
            if (!first.count(key)) first[key] = e;
            ++count[key];
        }
        std::vector<int> rep(t, -1), mode_rep(q, -1), partner(q, -1);
        std::vector<std::map<int, std::vector<int>>> group(p);  // per tensor: rep edge -> its modes, edge order
        for (int e = 0; e < t; ++e) {
            const int u = N.edges[2 * e], v = N.edges[2 * e + 1];
            const int a = owner[u], c = owner[v];
            if (a == c) {
                partner[u] = v;
                partner[v] = u;
                continue;
            }
            const std::pair<int, int> key{std::min(a, c), std::max(a, c)};
            if (count[key] < 2) continue;
            rep[e] = first[key];
            mode_rep[u] = mode_rep[v] = rep[e];
            group[a][rep[e]].push_back(u);
            group[c][rep[e]].push_back(v);
        }
        NormNet& nn = nb.nets[b];
        nn.X.assign(N.X, N.X + p);
        nn.dims.assign(p, {});
        nn.job.assign(p, -1);
        std::vector<int> new_id(q, -1);
        int nid = 0;
        for (int k = 0; k < p; ++k) {
            const tnsk_tensor& X = N.X[k];
            std::vector<int64_t> str(X.order);  // row-major strides of the source
            int64_t s = 1;
            for (int d = X.order - 1; d >= 0; --d) str[d] = s, s *= X.dims[d];
            std::vector<int> flat;  // kept modes in their new order
            bool traced = false;
            for (int g = moff[k]; g < moff[k + 1]; ++g) {
                if (partner[g] >= 0) {
                    traced = true;
                    continue;
                }
                const int r = mode_rep[g];
                if (r >= 0) {
                    const std::vector<int>& ms = group[k][r];
                    if (g != *std::min_element(ms.begin(), ms.end())) continue;
                    int64_t n = 1;
                    for (int x : ms) {
                        flat.push_back(x);
                        n *= dimg[x];
                        if (n > std::numeric_limits<int32_t>::max()) {
                            why = "network " + std::to_string(b) + ": merged contraction (WLOG 3) above 2^31 - 1";
                            return TNSK_ERR_UNSUPPORTED;
                        }
                    }
                    new_id[ms[0]] = nid++;
                    nn.dims[k].push_back(n);
                } else {
                    flat.push_back(g);
                    new_id[g] = nid++;
                    nn.dims[k].push_back(dimg[g]);
                }
            }
            const bool moved = !std::is_sorted(flat.begin(), flat.end());
            const bool reshaped = (int)nn.dims[k].size() != X.order;
            if (X.rung && (traced || moved || reshaped)) {
                why = "network " + std::to_string(b) + ": tensor " + std::to_string(k) +
                      " is a grouped (rung) tensor and would need a trace or reshape (WLOG 2/3)";
                return TNSK_ERR_UNSUPPORTED;
            }
            nn.X[k].order = (int32_t)nn.dims[k].size();
            if (!traced && !moved) continue;  // same data, at most a reshape
            NormJob J{};
            J.src = X.data;
            J.src_dtype = X.dtype;
            J.dst_f64 = X.dtype == TNSK_F64;
            J.n = (int32_t)flat.size();
            J.numel = 1;
            for (int j = 0; j < J.n; ++j) {
                J.dim[j] = dimg[flat[j]];
                J.str[j] = str[flat[j] - moff[k]];
                J.numel *= J.dim[j];
            }
            for (int g = moff[k]; g < moff[k + 1]; ++g)
                if (partner[g] > g) {
                    J.ddim[J.nd] = dimg[g];
                    J.dstr[J.nd] = str[g - moff[k]] + str[partner[g] - moff[k]];
                    ++J.nd;
                }
            nn.X[k].dtype = J.dst_f64 ? TNSK_F64 : TNSK_F32;
            nn.job[k] = (int)nb.jobs.size();
            nb.dst_off.push_back(off);
            off += ((size_t)J.numel * (J.dst_f64 ? 8 : 4) + 255) / 256 * 256;
            nb.most = std::max(nb.most, J.numel);
            nb.jobs.push_back(J);
        }
        for (int e = 0; e < t; ++e) {
            const int u = N.edges[2 * e], v = N.edges[2 * e + 1];
            if (owner[u] == owner[v] || (rep[e] >= 0 && rep[e] != e)) continue;
            nn.edges.push_back(new_id[u]);
            nn.edges.push_back(new_id[v]);
        }
        for (int k = 0; k < p; ++k) nn.X[k].dims = nn.dims[k].empty() ? nullptr : nn.dims[k].data();
        nn.net = N;
        nn.net.X = nn.X.data();
        nn.net.t = (int32_t)(nn.edges.size() / 2);
        nn.net.edges = nn.edges.empty() ? nullptr : nn.edges.data();
        nb.view[b] = nn.net;
        nb.used = true;
    }
    nb.desc_off = off;
    nb.bytes = off + nb.jobs.size() * sizeof(NormJob);
    return TNSK_OK;
}

}  // namespace tnsk

extern "C" tnsk_status tnsk_rewrite(const tnsk_network* net, const tnsk_params* params, int32_t cap_tensors,
                                    int32_t* p_out, int32_t* order_out, int32_t* copy_out, int64_t cap_dims,
                                    int64_t* dims_out, int32_t cap_edges, int32_t* t_out, int32_t* edges_out) {
    if (!net || !params || !p_out || !t_out || (cap_tensors > 0 && (!order_out || !copy_out)) ||
        (cap_dims > 0 && !dims_out) || (cap_edges > 0 && !edges_out))
        return TNSK_ERR_INVALID;
    tnsk::NormBatch nb;
    std::string why;
    const tnsk_status st = tnsk::normalize_batch(1, net, params, nb, why);
    if (st != TNSK_OK) return st;
    const tnsk_network& V = nb.view.empty() ? *net : nb.view[0];
    if (V.p < 0 || V.t < 0 || (V.p > 0 && !V.X) || (V.t > 0 && !V.edges)) return TNSK_ERR_INVALID;
    if (V.p > cap_tensors || V.t > cap_edges) return TNSK_ERR_INVALID;
    int64_t o = 0;
    for (int k = 0; k < V.p; ++k) {
        const tnsk_tensor& X = V.X[k];
        if (X.order < 0 || (X.order > 0 && !X.dims) || o + X.order > cap_dims) return TNSK_ERR_INVALID;
        order_out[k] = X.order;
        copy_out[k] = !nb.diag.empty() && !nb.diag[0].empty() ? nb.diag[0][(size_t)k] : 0;
        for (int d = 0; d < X.order; ++d) dims_out[o++] = X.dims[d];
    }
    for (int e = 0; e < 2 * V.t; ++e) edges_out[e] = V.edges[e];
    *p_out = V.p;
    *t_out = V.t;
    return TNSK_OK;
}

namespace tnsk {

void normalize_bind(NormBatch& nb, unsigned char* base) {
    for (size_t j = 0; j < nb.jobs.size(); ++j) nb.jobs[j].dst = base + nb.dst_off[j];
    for (size_t b = 0; b < nb.nets.size(); ++b) {
        NormNet& nn = nb.nets[b];
        for (size_t k = 0; k < nn.job.size(); ++k)
            if (nn.job[k] >= 0) nn.X[k].data = nb.jobs[(size_t)nn.job[k]].dst;
    }
}

}  // namespace tnsk
