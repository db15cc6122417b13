"""Join-size estimation as tensor network contraction (Sec. 5.1, Corollary
"multi-join-card-est"): the frequency tensor of each relation over its join columns is
a tensor of the network and every equi-join condition is a contraction between two
of their modes. A join class of three or more columns makes some mode part of two
contractions (a hyperedge); the library turns such classes into diagonal copy tensors
itself (WLOG 1). Frequency tensors are never stored: they start as all zeros in a
turnstile stream and receive one +1 per tuple as an update, so sketching costs
O(tuples) per repetition.

This module only lays out the network and the update lists (host bookkeeping); the
sketching, transform, product and combination run in libtnsk's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class JoinNetwork:
    shapes: list          # per relation: the dims of its joined columns (column order)
    edges: list           # contractions, pairs of global mode ids (hyperedges allowed)
    updates: list         # per relation: int64 flat entry indices of its tuples (value 1 each)
    n_relations: int


def join_network(relations, equalities, domains=None) -> JoinNetwork:
    """relations: list of int arrays [N_k, c_k] (tuples, values >= 0); equalities: list
    of ((k1, col1), (k2, col2)) equi-join conditions, each one contraction. Columns that
    join nothing are summed out (dropped from the frequency tensor). domains: optional
    {(k, col): size} (else the largest value in the class + 1)."""
    # union-find over (relation, column): a class shares one domain size
    parent = {}

    def find(x):
        parent.setdefault(x, x)
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b in equalities:
        parent[find(tuple(a))] = find(tuple(b))
    classes = {}
    for x in list(parent):
        classes.setdefault(find(x), []).append(x)
    size = {}
    for cl in classes.values():
        n = 0
        for k, c in cl:
            col = np.asarray(relations[k])[:, c]
            n = max(n, int(col.max()) + 1 if col.size else 1)
            if domains and (k, c) in domains:
                n = max(n, int(domains[(k, c)]))
        for x in cl:
            size[x] = n
    # tensors: each relation over its joined columns, in column order
    cols = [sorted(c for (k, c) in size if k == kk) for kk in range(len(relations))]
    shapes = [[size[(k, c)] for c in cols[k]] for k in range(len(relations))]
    off = [0]
    for sh in shapes:
        off.append(off[-1] + len(sh))
    mode = {(k, c): off[k] + cols[k].index(c) for k in range(len(relations)) for c in cols[k]}
    edges = [(mode[tuple(a)], mode[tuple(b)]) for a, b in equalities]
    updates = []
    for k, rel in enumerate(relations):
        rel = np.asarray(rel, dtype=np.int64)
        flat = np.zeros(rel.shape[0], dtype=np.int64)
        for c in cols[k]:
            flat = flat * size[(k, c)] + rel[:, c]
        updates.append(flat)
    return JoinNetwork(shapes, edges, updates, len(relations))


def exact_dense_tensors(jn: JoinNetwork):
    """The frequency tensors as dense FP64 arrays (small cases: tests, oracle)."""
    out = []
    for sh, flat in zip(jn.shapes, jn.updates):
        t = np.zeros(int(np.prod(sh)) if sh else 1)
        np.add.at(t, flat, 1.0)
        out.append(t.reshape(sh))
    return out
