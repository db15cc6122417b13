"""Oracle pins for method 2 (Sec. 4.4: Eq. 2, Alg. 2, Alg. 4, Alg. 5)."""
import json
import os
from functools import reduce

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ex(name):
    with open(os.path.join(GOLDEN, "paper_examples.json")) as f:
        return json.load(f)[name]


def _cs_matrix(bins, signs, m):
    C = np.zeros((m, len(bins)))
    C[bins, np.arange(len(bins))] = signs
    return C


def _F(m):
    j = np.arange(m)
    return np.exp(-2j * np.pi * np.outer(j, j) / m)


def _tensor_sketch2(Ca, Cb, m):
    """Def. "Tensor sketch" of order 2: T = F^{-1}((F Ca) . (F Cb)), m x m^2."""
    F = _F(m)
    rk = np.einsum("ja,jb->jab", F @ Ca, F @ Cb).reshape(m, -1)
    T = np.linalg.inv(F) @ rk
    assert np.allclose(T.imag, 0, atol=1e-9)
    return T.real


def _tree(X, edges, root):
    """Rooted tree of the footnote to Gamma(k): children in the order of k's modes."""
    off = np.concatenate([[0], np.cumsum([x.ndim for x in X])])
    owner = {g: k for k in range(len(X)) for g in range(off[k], off[k + 1])}
    partner = {}
    for e, (u, v) in enumerate(edges):
        partner[u] = (v, e)
        partner[v] = (u, e)
    children = {k: [] for k in range(len(X))}
    parent_mode = {root: None}
    stack = [root]
    while stack:
        k = stack.pop()
        for g in range(off[k], off[k + 1]):
            other, e = partner[g]
            l = owner[other]
            if l in parent_mode and parent_mode[l] is not None and parent_mode[l][0] == other:
                continue
            if l in parent_mode:
                continue
            parent_mode[l] = (other, e, other - off[l])
            children[k].append((l, g - off[k], e))
            stack.append(l)
    return children, parent_mode


def _recursive_sketch(k, children, X, edges, seed, r, m):
    """Def. "Recursive sketch": R = Q_2 Q_4 ... Q_qt S, S = (x) C_i (padding slots
    embed e_1, footnote), Q_l = T_{l,1} (x) ... (x) T_{l,l/2}."""
    ch = children[k]
    c = len(ch)
    if c == 0:
        return np.ones((1, 1))
    qt = 1
    while qt < c:
        qt *= 2
    dims = [d for x in X for d in x.shape]
    facs = []
    for j in range(qt):
        if j < c:
            l, mode, e = ch[j]
            b, s = oracle.count_sketch(seed, r, oracle.tid(2, e), dims[edges[e][0]], m)
            facs.append(_cs_matrix(b, s, m))
        else:
            b, s = oracle.count_sketch(seed, r, oracle.tid(3, k, j), 1, m)
            facs.append(_cs_matrix(b, s, m))  # C_pad e_1 as an m x 1 factor
    R = reduce(np.kron, facs)
    l = qt
    while l >= 2:
        Ts = []
        for j in range(l // 2):
            ba, sa = oracle.count_sketch(seed, r, oracle.tid(4, k, int(np.log2(l)), j, 0), m, m)
            bb, sb = oracle.count_sketch(seed, r, oracle.tid(4, k, int(np.log2(l)), j, 1), m, m)
            Ts.append(_tensor_sketch2(_cs_matrix(ba, sa, m), _cs_matrix(bb, sb, m), m))
        R = reduce(np.kron, Ts) @ R
        l //= 2
    return R


def _eq2(X, edges, root, seed, r, m):
    """Eq. 2 with every R_k materialised: y = vec(X_o)^T R_o^T R_o g(o),
    g(k) = (x)_{l in Gamma(k)} mat(X_l) R_l^T R_l g(l), g(leaf) = 1."""
    children, pmode = _tree(X, edges, root)
    Rs = {k: _recursive_sketch(k, children, X, edges, seed, r, m) for k in range(len(X))}

    def g(k):
        parts = []
        for l, _, _ in children[k]:
            d = pmode[l][2]
            M = np.moveaxis(X[l], d, 0).reshape(X[l].shape[d], -1)  # mat(X_l), parent mode first
            parts.append(M @ Rs[l].T @ Rs[l] @ g(l))
        return reduce(np.kron, parts) if parts else np.ones(1)

    return float(X[root].ravel() @ Rs[root].T @ Rs[root] @ g(root))


def _example5(n, rng):
    ex = _ex("example5")
    X = [rng.standard_normal((n,) * q) for q in ex["orders"]]
    edges = [(u - 1, v - 1) for u, v in ex["edges"]]
    return ex, X, edges


def test_example5_tree_structure():
    ex, X, edges = _example5(2, np.random.default_rng(0))
    children, _ = _tree(X, edges, ex["root"] - 1)
    for k, ch in ex["children"].items():
        assert [l + 1 for l, _, _ in children[int(k) - 1]] == ch
    for k, q in ex["recursive_sketch_order"].items():
        assert len(children[int(k) - 1]) == q


@pytest.mark.parametrize("n,m,root", [(2, 4, 0), (3, 8, 0), (2, 8, 3), (2, 4, 6)])
def test_alg2_equals_eq2_with_materialised_recursive_sketches(n, m, root):
    rng = np.random.default_rng(10 * n + m + root)
    ex, X, edges = _example5(n, rng)
    R, seed = 3, 77
    y, s = oracle.m2_estimate(X, edges, m=m, reps=R, seed=seed, root=root)
    for r in range(R):
        want = _eq2(X, edges, root, seed, r, m)
        assert np.isclose(y[r], want, rtol=1e-9, atol=1e-9 * s[r])
        assert s[r] >= abs(y[r]) - 1e-12


def test_exact_on_paths_with_injective_count_sketches():
    # A path rooted at an end: every R_k is one count sketch (order 1, no Q). With
    # injective C and unit signs, C^T C = I, so Eq. 2 reduces to the recursion of
    # Lemma "recursive-AFTNC": the estimate is exact. The middle tensor's parent
    # mode is its second mode (the footnote's permutation is handled logically).
    rng = np.random.default_rng(1)
    X = [rng.standard_normal(3), rng.standard_normal((4, 3)), rng.standard_normal((4, 5)), rng.standard_normal(5)]
    edges = [(0, 2), (1, 3), (4, 5)]
    m = 8
    eb = np.concatenate([np.arange(3), np.arange(4), np.arange(5)])[None, :]
    es = np.ones_like(eb, dtype=np.int8)
    y, _ = oracle.m2_estimate(X, edges, m=m, reps=1, seed=0, root=0, edge_bins=eb, edge_signs=es)
    assert np.isclose(y[0], oracle.tc_einsum(X, edges, []), rtol=1e-12)
    # the same holds from the other end of the path
    y, _ = oracle.m2_estimate(X, edges, m=m, reps=1, seed=0, root=3, edge_bins=eb, edge_signs=es)
    assert np.isclose(y[0], oracle.tc_einsum(X, edges, []), rtol=1e-12)


def test_unbiased_and_within_variance_bound():
    # Lemma "acyclic-expectation-variance": E[y] = tc, Var <= ((1+8/m)^{2t} - 1) prod ||X_k||^2
    rng = np.random.default_rng(2)
    ex, X, edges = _example5(3, rng)
    m, R = 32, 6000
    y, _ = oracle.m2_estimate(X, edges, m=m, reps=R, seed=5, root=0)
    tc = oracle.tc_einsum(X, edges, [])
    assert abs(y.mean() - tc) <= 5 * y.std() / np.sqrt(R)
    bound = ((1 + 8 / m) ** (2 * len(edges)) - 1) * oracle.frobenius_product(X) ** 2
    assert y.var() <= bound * (1 + 5 * np.sqrt(2 / R))


def test_rejects_cycles_open_legs_and_forests():
    rng = np.random.default_rng(3)
    A = [rng.standard_normal((3, 3)) for _ in range(3)]
    with pytest.raises(oracle.OracleError) as e:
        oracle.m2_estimate(A, [(1, 2), (3, 4), (5, 0)], m=8, reps=1, seed=1)
    assert e.value.status == oracle.ORC_CYCLIC
    with pytest.raises(oracle.OracleError) as e:  # two contractions between one pair (WLOG 3)
        oracle.m2_estimate(A[:2], [(0, 2), (1, 3)], m=8, reps=1, seed=1)
    assert e.value.status == oracle.ORC_CYCLIC
    with pytest.raises(oracle.OracleError) as e:  # a trace inside one tensor (WLOG 2)
        oracle.m2_estimate(A[:1], [(0, 1)], m=8, reps=1, seed=1)
    assert e.value.status == oracle.ORC_CYCLIC
    x = [rng.standard_normal(3) for _ in range(4)]
    with pytest.raises(oracle.OracleError) as e:
        oracle.m2_estimate(x, [(0, 1), (2, 3)], m=8, reps=1, seed=1)
    assert e.value.status == oracle.ORC_UNSUPPORTED


def test_scalar_root():
    y, _ = oracle.m2_estimate([np.array(4.0)], [], m=8, reps=2, seed=1)
    assert np.allclose(y, 4.0)
