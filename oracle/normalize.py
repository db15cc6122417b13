"""WLOG 1, WLOG 2 and WLOG 3 of Sec. 4.1 in FP64 numpy (test infrastructure only: the
tests, the smoke check and the benchmark's CPU-baseline leg are the only callers).

``copy_tensors`` (WLOG 1) replaces each class of three or more modes that
contractions force equal (a mode in several contractions) by a diagonal copy tensor
joined to every member; it is the form the general method takes such networks in.

The acyclic method (Sec. 4.4) assumes that every contraction joins two different
tensors and that at most one contraction joins any two tensors. A network that
breaks either assumption is first rewritten into one with the same contraction
value:

* WLOG 2: a contraction (u, v) whose modes belong to the same tensor X_k is summed
  exactly, X'_k(..) = sum_i X_k(.., i, .., i, ..), and both modes leave X_k;
* WLOG 3: the r >= 2 contractions e_1 < ... < e_r (by position in the edge list)
  between a pair of tensors become one contraction by reshaping both tensors: in
  each of them the r modes are replaced by a single mode, placed where the first
  of them (the lowest mode id in that tensor) was, of size n_{e_1} ... n_{e_r},
  whose index is row-major over (i_{e_1}, ..., i_{e_r}). The paper's example, two
  matrices joined on both modes, becomes the inner product of vec(A) and vec(B).

Tensors keep their order and count; the other modes keep their relative order;
the remaining contractions keep their order, a merged one standing where e_1
stood, with the endpoint in e_1's first tensor first. Open modes are renumbered
with the rest. The rewrite is written with numpy einsum (a repeated subscript
sums a diagonal), transpose and reshape.
"""
from __future__ import annotations

import string

import numpy as np


def copy_tensors(tensors, edges, open_modes=()):
    """WLOG 1 of Sec. 4.1: a mode in several contractions gets virtual copies. The modes
    linked by contractions fall into classes whose indices must all agree; a class of
    three or more modes becomes a diagonal copy tensor delta(i, ..., i) of order d
    (one mode per class member) joined to each member. Returns (tensors', edges',
    open') with: the original tensors, then one copy tensor per such class (classes
    ordered by their lowest mode id); first the contractions of two-mode classes in
    their original order (a repeated pair kept once), then per copy tensor the
    contractions (g_j, c_j) for the class's modes g_1 < ... < g_d and the copy
    tensor's modes c_j in order. Mode ids of the original tensors do not change."""
    tensors = [np.asarray(x, dtype=np.float64) for x in tensors]
    dims = [d for x in tensors for d in x.shape]
    q = len(dims)
    parent = list(range(q))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for u, v in edges:
        parent[find(u)] = find(v)
    members = {}
    for u, v in edges:
        for g in (u, v):
            members.setdefault(find(g), set()).add(g)
    out_t, out_e, seen = list(tensors), [], set()
    for u, v in edges:
        cl = members[find(u)]
        if len(cl) == 2 and frozenset(cl) not in seen:
            seen.add(frozenset(cl))
            out_e.append((u, v))
    nxt = q
    for cl in sorted((sorted(c) for c in members.values() if len(c) >= 3), key=lambda c: c[0]):
        d, n = len(cl), dims[cl[0]]
        delta = np.zeros((n,) * d)
        for i in range(n):
            delta[(i,) * d] = 1.0
        out_t.append(delta)
        for j, g in enumerate(cl):
            out_e.append((g, nxt + j))
        nxt += d
    return out_t, out_e, list(open_modes)


def needs_normalize(tensors, edges) -> bool:
    """True when a contraction lies inside one tensor or two join the same pair."""
    owner = _owner(tensors)
    seen = set()
    for u, v in edges:
        a, b = owner[u], owner[v]
        if a == b:
            return True
        key = (min(a, b), max(a, b))
        if key in seen:
            return True
        seen.add(key)
    return False


def _owner(tensors):
    own = []
    for k, x in enumerate(tensors):
        own += [k] * np.ndim(x)
    return own


def normalize(tensors, edges, open_modes=()):
    """(tensors', edges', open') of the rewritten network (FP64 arrays)."""
    tensors = [np.asarray(x, dtype=np.float64) for x in tensors]
    owner = _owner(tensors)
    off = [0]
    for x in tensors:
        off.append(off[-1] + x.ndim)
    # WLOG 3 groups: pair of tensors -> its edges in list order
    groups = {}
    for e, (u, v) in enumerate(edges):
        a, b = owner[u], owner[v]
        if a != b:
            groups.setdefault((min(a, b), max(a, b)), []).append(e)
    merged_into = {}  # edge -> first edge of its group (groups of two or more)
    for es in groups.values():
        if len(es) >= 2:
            for e in es:
                merged_into[e] = es[0]
    # per tensor: the new mode list; each entry is a tuple of old mode ids
    new_modes = []
    for k, x in enumerate(tensors):
        mine = range(off[k], off[k + 1])
        traced = set()
        group_modes = {}  # first edge -> this tensor's modes of the group, in edge order
        for e, (u, v) in enumerate(edges):
            if owner[u] == k and owner[v] == k:
                traced |= {u, v}
            elif e in merged_into:
                g = u if owner[u] == k else v if owner[v] == k else None
                if g is not None:
                    group_modes.setdefault(merged_into[e], []).append(g)
        first_of = {min(ms): f for f, ms in group_modes.items()}
        in_group = {g for ms in group_modes.values() for g in ms}
        modes = []
        for g in mine:
            if g in traced:
                continue
            if g in first_of:
                modes.append(tuple(group_modes[first_of[g]]))
            elif g not in in_group:
                modes.append((g,))
        new_modes.append(modes)
    # the rewritten tensors: einsum over the diagonals and into the new order, then reshape
    out_tensors = []
    for k, x in enumerate(tensors):
        letters = {}
        nxt = iter(string.ascii_letters)
        sub = []
        for g in range(off[k], off[k + 1]):
            if g not in letters:
                letters[g] = next(nxt)
            sub.append(letters[g])
        for u, v in edges:  # a traced pair shares one letter
            if owner[u] == k and owner[v] == k:
                sub[v - off[k]] = sub[u - off[k]]
        flat = [g for ms in new_modes[k] for g in ms]
        y = np.einsum("".join(sub) + "->" + "".join(letters[g] for g in flat), x)
        shape = [int(np.prod([x.shape[g - off[k]] for g in ms])) for ms in new_modes[k]]
        out_tensors.append(y.reshape(shape).copy())  # C order, 0-d kept 0-d
    # new global ids: a new mode is named by its first old mode
    new_id, nid = {}, 0
    for k in range(len(tensors)):
        for ms in new_modes[k]:
            new_id[ms[0]] = nid
            nid += 1
    out_edges = []
    for e, (u, v) in enumerate(edges):
        if owner[u] == owner[v]:
            continue
        if e in merged_into and merged_into[e] != e:
            continue
        if e in merged_into:  # the group's representative: its modes are the groups' first modes
            a, b = owner[u], owner[v]
            mu = [ms[0] for ms in new_modes[a] if len(ms) > 1 and u in ms]
            mv = [ms[0] for ms in new_modes[b] if len(ms) > 1 and v in ms]
            out_edges.append((new_id[mu[0]], new_id[mv[0]]))
        else:
            out_edges.append((new_id[u], new_id[v]))
    out_open = [new_id[g] for g in open_modes]
    return out_tensors, out_edges, out_open
