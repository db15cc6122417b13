"""Exact tensor network contraction in FP64 (test infrastructure only).

Implements Def. "Tensor contraction" / "Tensor network contraction" (Sec. 1) of
"Approximating Tensor Network Contraction with Sketches" twice:

* ``tc_definition``   -- the Iverson-bracket sum written out: every global
  multi-index i over all modes, weight prod_k X_k(i_k) * prod_{(u,v) in E} [i_u = i_v].
  Tiny networks only.
* ``tc_reduced``      -- the same sum after reducing the brackets (as in Example 1):
  one index value per contraction plus the open indices.
* ``tc_einsum``       -- the same sum evaluated by pairwise contractions (numpy einsum
  in float64, greedy order). Used where the sums above are infeasible; pinned to
  them on small networks by the tests.

Only tests, the smoke check and the benchmark's CPU-baseline leg use this module.
"""
from __future__ import annotations

import itertools

import numpy as np


def _modes(tensors):
    off = [0]
    for x in tensors:
        off.append(off[-1] + np.ndim(x))
    dims = [d for x in tensors for d in np.shape(x)]
    return off, dims


def tc_definition(tensors, edges, open_modes):
    """Literal Def. "Tensor contraction" applied to X_1 x ... x X_p (Def. "TNC")."""
    tensors = [np.asarray(x, dtype=np.float64) for x in tensors]
    off, dims = _modes(tensors)
    out_shape = tuple(dims[g] for g in open_modes)
    out = np.zeros(out_shape, dtype=np.float64)
    for i in itertools.product(*[range(d) for d in dims]):
        if not all(i[u] == i[v] for u, v in edges):
            continue
        w = 1.0
        for k, x in enumerate(tensors):
            w *= float(x[tuple(i[off[k]:off[k + 1]])])
        out[tuple(i[g] for g in open_modes)] += w
    return out


def tc_reduced(tensors, edges, open_modes):
    """Def. "Tensor contraction" with the Iverson brackets reduced: one value per
    contraction (u, v) shared by both modes, open modes free."""
    tensors = [np.asarray(x, dtype=np.float64) for x in tensors]
    off, dims = _modes(tensors)
    q = len(dims)
    label = [None] * q  # which free variable indexes each mode
    for e, (u, v) in enumerate(edges):
        label[u] = ("e", e)
        label[v] = ("e", e)
    for j, g in enumerate(open_modes):
        label[g] = ("o", j)
    e_dims = [dims[u] for u, _ in edges]
    o_dims = [dims[g] for g in open_modes]
    out = np.zeros(tuple(o_dims), dtype=np.float64)
    for ev in itertools.product(*[range(d) for d in e_dims]):
        for ov in itertools.product(*[range(d) for d in o_dims]):
            w = 1.0
            for k, x in enumerate(tensors):
                idx = []
                for g in range(off[k], off[k + 1]):
                    kind, a = label[g]
                    idx.append(ev[a] if kind == "e" else ov[a])
                w *= float(x[tuple(idx)])
            out[tuple(ov)] += w
    return out


def tc_einsum(tensors, edges, open_modes):
    """Def. "Tensor contraction" evaluated by pairwise contractions in float64."""
    tensors = [np.asarray(x, dtype=np.float64) for x in tensors]
    off, dims = _modes(tensors)
    q = len(dims)
    lab = [-1] * q
    nxt = 0
    for u, v in edges:
        lab[u] = lab[v] = nxt
        nxt += 1
    for g in open_modes:
        lab[g] = nxt
        nxt += 1
    if nxt > 52:
        raise ValueError("network has more than 52 distinct indices")
    args = []
    for k, x in enumerate(tensors):
        args.append(x)
        args.append([lab[g] for g in range(off[k], off[k + 1])])
    args.append([lab[g] for g in open_modes])
    return np.asarray(np.einsum(*args, optimize="greedy"), dtype=np.float64)


def tc_sequential(tensors, edges, open_modes):
    """Def. "Tensor contraction" evaluated by absorbing the tensors one at a time, in
    the given order, into a running tensor (float64); an index is summed as soon as
    no later tensor carries it and it is not open. On a grid in row-major order the
    running tensor holds at most one row of bonds."""
    tensors = [np.asarray(x, dtype=np.float64) for x in tensors]
    off, dims = _modes(tensors)
    q = len(dims)
    lab = list(range(q))  # unmatched modes keep their own label
    for u, v in edges:
        lab[v] = lab[u]
    open_labels = [lab[g] for g in open_modes]
    owner = [[lab[g] for g in range(off[k], off[k + 1])] for k in range(len(tensors))]
    if not tensors:
        return np.asarray(1.0)
    run, run_lab = tensors[0], owner[0]
    keep = lambda labels, k: [l for i, l in enumerate(labels) if l not in labels[:i] and
                              (l in open_labels or any(l in owner[j] for j in range(k + 1, len(tensors))))]
    out = keep(run_lab, 0)
    run = np.einsum(run, run_lab, out)
    run_lab = out
    for k in range(1, len(tensors)):
        out = keep(run_lab + owner[k], k)
        run = np.einsum(run, run_lab, tensors[k], owner[k], out)
        run_lab = out
    return np.asarray(np.einsum(run, run_lab, open_labels), dtype=np.float64)


def frobenius_product(tensors):
    """||X||_F of the tensor product = prod_k ||X_k||_F (proof of Theorem 1)."""
    return float(np.prod([np.linalg.norm(np.asarray(x, dtype=np.float64).ravel()) for x in tensors]))
