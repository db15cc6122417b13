"""Seeded synthetic tensor networks (inputs only; none of the estimators' arithmetic).

Every generator takes a seed and returns a ``NetSpec``: float64 numpy tensors
(row-major), contractions as pairs of global 0-based mode ids (numbered across
X_1..X_p in order, as in Def. "Tensor product" / Example 1 of the paper) and the
open-mode output order. ``to_torch`` moves a spec to the GPU in a given dtype.

Workloads (shapes and distributions of the benchmark configurations):
  triangle      three n x n N(0,1) matrices, full contraction tr(ABC)
  tt_cores      two tensor trains (bond 32, physical 8, N(0, 1/sqrt(32)))
  tt_ladder     the two trains with physical legs contracted pairwise (cyclic)
  tt_chain      the same value as an acyclic chain: each site's pair A_k x B_k with
                the physical leg summed and the two bonds merged into one mode
                (the paper's WLOG 2 and WLOG 3 reductions, Sec. 4.1)
  grid          L1 x L2 grid network, U(0,1) entries
  random_network  random connected graphs with degree, dimension and open-leg mixes
  random_tree   random acyclic networks
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DATA_SEED = 20260307
HASH_SEED = 0x7E57


@dataclass
class NetSpec:
    tensors: list
    edges: list
    open: list = field(default_factory=list)
    name: str = ""

    @property
    def p(self):
        return len(self.tensors)

    @property
    def t(self):
        return len(self.edges)

    def numel(self):
        return int(sum(np.asarray(x).size for x in self.tensors))


def _mode_offsets(shapes):
    off = [0]
    for s in shapes:
        off.append(off[-1] + len(s))
    return off


def triangle(n: int = 64, seed: int = DATA_SEED) -> NetSpec:
    rng = np.random.default_rng(seed)
    A, B, C = (rng.standard_normal((n, n)) for _ in range(3))
    # modes A=(0,1) B=(2,3) C=(4,5): tr(ABC) = tc(A x B x C, {(1,2),(3,4),(5,0)})
    return NetSpec([A, B, C], [(1, 2), (3, 4), (5, 0)], [], f"triangle{n}")


def tt_cores(sites: int = 8, bond: int = 32, phys: int = 8, seed: int = DATA_SEED, std: float | None = None):
    """Two tensor trains: end cores [phys, bond] / [bond, phys], inner [bond, phys, bond]."""
    rng = np.random.default_rng(seed)
    std = 1.0 / np.sqrt(bond) if std is None else std

    def train():
        cores = [rng.normal(0, std, (phys, bond))]
        cores += [rng.normal(0, std, (bond, phys, bond)) for _ in range(sites - 2)]
        cores.append(rng.normal(0, std, (bond, phys)))
        return cores

    return train(), train()


def tt_ladder(A, B) -> NetSpec:
    """Both trains as one network: bonds along each train, physical legs A_k-B_k."""
    sites = len(A)
    shapes = [a.shape for a in A] + [b.shape for b in B]
    off = _mode_offsets(shapes)

    def modes(k, train):  # (left bond, phys, right bond) global ids, None if absent
        base = off[k + (sites if train else 0)]
        if k == 0:
            return None, base, base + 1
        if k == sites - 1:
            return base, base + 1, None
        return base, base + 1, base + 2

    edges = []
    for train in (0, 1):
        for k in range(sites - 1):
            edges.append((modes(k, train)[2], modes(k + 1, train)[0]))
    for k in range(sites):
        edges.append((modes(k, 0)[1], modes(k, 1)[1]))
    return NetSpec(list(A) + list(B), edges, [], f"tt_ladder{sites}")


def tt_chain(A, B) -> NetSpec:
    """Acyclic chain with the ladder's value: M_k = sum_s A_k[., s, .] (x) B_k[., s, .],
    bond pairs (alpha, beta) merged into one index alpha * bond + beta."""
    sites = len(A)
    M = [np.einsum("sa,sb->ab", A[0], B[0]).reshape(-1)]
    for k in range(1, sites - 1):
        M.append(np.einsum("asc,bsd->abcd", A[k], B[k]).reshape(A[k].shape[0] * B[k].shape[0], -1))
    M.append(np.einsum("as,bs->ab", A[-1], B[-1]).reshape(-1))
    off = _mode_offsets([x.shape for x in M])
    edges = [(off[k + 1] - 1, off[k + 1]) for k in range(sites - 1)]
    return NetSpec(M, edges, [], f"tt_chain{sites}")


def grid(L1: int = 4, L2: int = 4, bond: int = 8, seed: int = DATA_SEED) -> NetSpec:
    """Grid network; a site's modes are its neighbours in the order up, left, right, down."""
    rng = np.random.default_rng(seed)
    nbrs = {}
    for i in range(L1):
        for j in range(L2):
            nb = []
            for di, dj in ((-1, 0), (0, -1), (0, 1), (1, 0)):
                a, b = i + di, j + dj
                if 0 <= a < L1 and 0 <= b < L2:
                    nb.append((a, b))
            nbrs[(i, j)] = nb
    sites = [(i, j) for i in range(L1) for j in range(L2)]
    tensors = [rng.uniform(0.0, 1.0, (bond,) * len(nbrs[s])) for s in sites]
    off = _mode_offsets([x.shape for x in tensors])
    index = {s: n for n, s in enumerate(sites)}
    edges = []
    for s in sites:
        for slot, nb in enumerate(nbrs[s]):
            if index[nb] > index[s]:
                back = nbrs[nb].index(s)
                edges.append((off[index[s]] + slot, off[index[nb]] + back))
    return NetSpec(tensors, edges, [], f"grid{L1}x{L2}b{bond}")


def random_network(rng, p_range=(4, 12), deg_range=(2, 4), dim_range=(2, 16), max_open=2,
                   open_dim_range=(2, 16), dist: str = "normal") -> NetSpec:
    """Random connected graph: a random spanning tree, then extra edges (no self loops,
    no parallel edges) while both ends are below their target degree; uniform edge
    dims; 0..max_open open legs on random tensors."""
    p = int(rng.integers(p_range[0], p_range[1] + 1))
    target = rng.integers(deg_range[0], deg_range[1] + 1, size=p)
    pairs = []
    deg = np.zeros(p, dtype=int)
    for k in range(1, p):
        j = int(rng.integers(0, k))
        pairs.append((j, k))
        deg[j] += 1
        deg[k] += 1
    present = set(pairs)
    while True:
        cand = [(a, b) for a in range(p) for b in range(a + 1, p)
                if (a, b) not in present and deg[a] < target[a] and deg[b] < target[b]]
        if not cand:
            break
        a, b = cand[int(rng.integers(0, len(cand)))]
        pairs.append((a, b))
        present.add((a, b))
        deg[a] += 1
        deg[b] += 1
    edim = [int(rng.integers(dim_range[0], dim_range[1] + 1)) for _ in pairs]
    n_open = int(rng.integers(0, max_open + 1))
    open_at = [int(rng.integers(0, p)) for _ in range(n_open)]
    open_dims = [int(rng.integers(open_dim_range[0], open_dim_range[1] + 1)) for _ in range(n_open)]
    # modes of tensor k: its edges in edge order, then its open legs
    slots = [[] for _ in range(p)]
    for e, (a, b) in enumerate(pairs):
        slots[a].append(("e", e))
        slots[b].append(("e", e))
    for j, k in enumerate(open_at):
        slots[k].append(("o", j))
    shapes = [tuple(edim[x] if kind == "e" else open_dims[x] for kind, x in sl) for sl in slots]
    off = _mode_offsets(shapes)
    ends = {}
    open_modes = [None] * n_open
    for k, sl in enumerate(slots):
        for d, (kind, x) in enumerate(sl):
            if kind == "e":
                ends.setdefault(x, []).append(off[k] + d)
            else:
                open_modes[x] = off[k] + d
    edges = [tuple(ends[e]) for e in range(len(pairs))]
    if dist == "normal":
        tensors = [rng.standard_normal(s) for s in shapes]
    else:
        tensors = [rng.uniform(0.0, 1.0, s) for s in shapes]
    return NetSpec(tensors, edges, open_modes, "random")


def random_tree(rng, p: int, dim_range=(2, 6), max_children: int = 3) -> NetSpec:
    """Random acyclic connected network (a random tree over p tensors)."""
    pairs = []
    kids = np.zeros(p, dtype=int)
    for k in range(1, p):
        choices = [j for j in range(k) if kids[j] < max_children] or list(range(k))
        j = int(choices[int(rng.integers(0, len(choices)))])
        pairs.append((j, k))
        kids[j] += 1
    edim = [int(rng.integers(dim_range[0], dim_range[1] + 1)) for _ in pairs]
    slots = [[] for _ in range(p)]
    for e, (a, b) in enumerate(pairs):
        slots[a].append(e)
        slots[b].append(e)
    for sl in slots:  # random mode order, so parents are not always mode 0
        rng.shuffle(sl)
    shapes = [tuple(edim[e] for e in sl) for sl in slots]
    off = _mode_offsets(shapes)
    ends = {}
    for k, sl in enumerate(slots):
        for d, e in enumerate(sl):
            ends.setdefault(e, []).append(off[k] + d)
    edges = [tuple(ends[e]) for e in range(len(pairs))]
    tensors = [rng.standard_normal(s) for s in shapes]
    return NetSpec(tensors, edges, [], f"tree{p}")


def to_torch(spec: NetSpec, device="cuda", dtype=None):
    """The spec's tensors as contiguous torch tensors (float32 by default)."""
    import torch

    dtype = torch.float32 if dtype is None else dtype
    # np.array (not ascontiguousarray) keeps 0-d scalars 0-d
    return [torch.as_tensor(np.array(x, dtype=np.float64)).to(device=device, dtype=dtype).contiguous()
            for x in spec.tensors]
