"""Oracle pins for method 1 (Sec. 4.2: Eq. 1, Alg. 1, complement count sketches)."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ex(name):
    with open(os.path.join(GOLDEN, "paper_examples.json")) as f:
        return json.load(f)[name]


def _cs_matrix(bins, signs, m):
    """Def. "Count sketch": C(j, i) = s(i) [h(i) = j]."""
    C = np.zeros((m, len(bins)))
    C[bins, np.arange(len(bins))] = signs
    return C


def _complement_matrix(bins, signs, m):
    """Def. "Complement count sketch" (0-based): C'(j, i) = s(i) [-h(i) = j mod m]."""
    return _cs_matrix((-np.asarray(bins)) % m, signs, m)


def _F(m):
    j = np.arange(m)
    return np.exp(-2j * np.pi * np.outer(j, j) / m)


def test_complement_lemma_and_involution():
    m, n = 16, 11
    b, s = oracle.count_sketch(4, 0, 1 << 56, n, m)
    x = np.random.default_rng(0).standard_normal(n)
    C, Cc = _cs_matrix(b, s, m), _complement_matrix(b, s, m)
    assert np.allclose(_F(m) @ (Cc @ x), np.conj(_F(m) @ (C @ x)))  # Lemma "complement-count-sketch"
    bb = (-((-b) % m)) % m  # (C')' = C (Remark)
    assert np.array_equal(bb, b)


def test_single_contraction_is_count_sketch_inner_product():
    # t = 1, X1 = x, X2 = y: Eq. 1 reduces to <Cx, Cy> (Lemma "count-sketch",
    # via e_1^T F^{-1}(x o conj(y)) = <x, y>/m in the proof of Lemma
    # "general-expectation-variance")
    rng = np.random.default_rng(1)
    n, m, R = 40, 16, 12
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    bins, signs = oracle.m1_tables([x, y], [(0, 1)], [], seed=3, reps=R, m=m)
    est, _ = oracle.m1_estimate([x, y], [(0, 1)], [], m=m, bins=bins, signs=signs)
    for r in range(R):
        C = _cs_matrix(bins[r], signs[r], m)
        assert np.isclose(est[r, 0], (C @ x) @ (C @ y), rtol=1e-12, atol=1e-12)


def test_sketch_equals_materialised_tensor_sketch():
    # Def. "Tensor sketch": T = F^{-1}((F C_1) . (F C_2) . (F C_3)) applied to vec(X),
    # with the complement on the second mode of an edge (Eq. 1, Alg. 1)
    rng = np.random.default_rng(2)
    m = 8
    X = rng.standard_normal((2, 3, 2))
    ys = [rng.standard_normal(2), rng.standard_normal(3), rng.standard_normal(2)]
    tensors = [X] + ys
    edges = [(0, 3), (4, 1), (2, 5)]  # mode 1 of X is the second mode of its edge
    bins, signs = oracle.m1_tables(tensors, edges, [], seed=7, reps=2, m=m)
    xs = oracle.m1_sketch(tensors, edges, [], m, bins, signs)
    off = np.concatenate([[0], np.cumsum([2, 3, 2])])
    F = _F(m)
    for r in range(2):
        Cs = [_cs_matrix(bins[r, off[0]:off[1]], signs[r, off[0]:off[1]], m),
              _complement_matrix(bins[r, off[1]:off[2]], signs[r, off[1]:off[2]], m),
              _cs_matrix(bins[r, off[2]:off[3]], signs[r, off[2]:off[3]], m)]
        FC = [F @ C for C in Cs]
        # row-wise Kronecker product (Def. "Row-wise Kronecker product")
        rk = np.einsum("ja,jb,jc->jabc", *FC).reshape(m, -1)
        T = np.linalg.inv(F) @ rk
        assert np.allclose(T.imag, 0, atol=1e-10)
        assert np.allclose(xs[r, :m], T.real @ X.ravel(), atol=1e-10)


def _mixed_radix_tables(edge_dims, m):
    bins, w = [], 1
    for n in edge_dims:
        bins.append(np.arange(n) * w)
        w *= n
    assert w <= m
    b = np.concatenate(bins)[None, :]
    return b.astype(np.int64), np.ones_like(b, dtype=np.int8)


@pytest.mark.parametrize("case", ["triangle", "open_legs", "self_contraction"])
def test_exact_when_bins_are_mixed_radix(case):
    # With signs +1 and h_e(i) = i * prod_{e'<e} n_e', m >= prod n_e, the bracket
    # [sum_e h_e(i_u) - h_e(i_v) = 0 mod m] in the expansion of the proof of Lemma
    # "general-expectation-variance" equals prod_e [i_u = i_v]: the estimate is tc.
    rng = np.random.default_rng(3)
    if case == "triangle":
        X = [rng.standard_normal((3, 2)), rng.standard_normal((2, 4)), rng.standard_normal((4, 3))]
        edges, open_modes = [(1, 2), (3, 4), (5, 0)], []
    elif case == "open_legs":
        X = [rng.standard_normal((3, 2, 2)), rng.standard_normal((2, 3)), rng.standard_normal((3, 3))]
        edges, open_modes = [(1, 3), (4, 5)], [6, 0, 2]
    else:
        X = [rng.standard_normal((3, 2, 3)), rng.standard_normal(2)]
        edges, open_modes = [(0, 2), (1, 3)], []
    dims = [d for x in X for d in x.shape]
    edge_dims = [dims[u] for u, _ in edges]
    W = int(np.prod(edge_dims))
    m = 1 << int(np.ceil(np.log2(max(W, 1))))
    b, s = _mixed_radix_tables(edge_dims, m)
    y, _ = oracle.m1_estimate(X, edges, open_modes, m=m, bins=b, signs=s)
    want = oracle.tc_einsum(X, edges, open_modes).ravel()
    assert np.allclose(y[0], want, atol=1e-10)


def _brute_expansion(X, edges, m, bins, signs):
    """sum_i prod_k X_k(i_k) prod_e s_e(i_u) s_e(i_v) [sum_e h_e(i_u) - h_e(i_v) = 0 mod m],
    the expansion of Eq. 1 in the proof of Lemma "general-expectation-variance"."""
    dims = [d for x in X for d in x.shape]
    off = np.concatenate([[0], np.cumsum([x.ndim for x in X])])
    eoff = np.concatenate([[0], np.cumsum([dims[u] for u, _ in edges])])
    total = 0.0
    for i in itertools.product(*[range(d) for d in dims]):
        w = 1.0
        for k, x in enumerate(X):
            w *= x[tuple(i[off[k]:off[k + 1]])]
        sg, h = 1, 0
        for e, (u, v) in enumerate(edges):
            sg *= signs[eoff[e] + i[u]] * signs[eoff[e] + i[v]]
            h += bins[eoff[e] + i[u]] - bins[eoff[e] + i[v]]
        if h % m == 0:
            total += sg * w
    return total


def test_fft_form_time_domain_and_brute_expansion_agree():
    ex = _ex("example4")
    rng = np.random.default_rng(4)
    X = [rng.standard_normal((3, 3)) for _ in range(3)]
    edges = [(u - 1, v - 1) for u, v in ex["edges"]]
    assert [u + 1 for u, _ in edges] == ex["count_sketch_modes"]
    assert [v + 1 for _, v in edges] == ex["complement_modes"]
    m, R = 8, 3
    bins, signs = oracle.m1_tables(X, edges, [], seed=5, reps=R, m=m)
    y, s = oracle.m1_estimate(X, edges, [], m=m, bins=bins, signs=signs)
    xs = oracle.m1_sketch(X, edges, [], m, bins, signs)
    for r in range(R):
        # time domain: (x_1 * x_2 * x_3)_0 by Def. "Circular convolution" (Lemma "conv-thm")
        c = xs[r, 0:m]
        for k in (1, 2):
            xk = xs[r, k * m:(k + 1) * m]
            c = np.array([sum(c[i] * xk[(j - i) % m] for i in range(m)) for j in range(m)])
        assert np.isclose(y[r, 0], c[0], rtol=1e-12, atol=1e-12)
        assert np.isclose(y[r, 0], _brute_expansion(X, edges, m, bins[r], signs[r]), rtol=1e-12, atol=1e-12)
        assert s[r, 0] >= abs(y[r, 0]) - 1e-12


def test_open_entries_equal_full_estimates_of_subtensors():
    # Corollary "full-to-partial-tc": each output entry is the full estimator on
    # the subtensors with the open indices fixed (same sketches)
    rng = np.random.default_rng(6)
    X = [rng.standard_normal((3, 4)), rng.standard_normal((4, 5, 2)), rng.standard_normal((5, 3))]
    edges = [(1, 2), (3, 5), (6, 0)]  # modes: X0=(0,1), X1=(2,3,4), X2=(5,6)
    open_modes = [4]
    m, R = 16, 4
    bins, signs = oracle.m1_tables(X, edges, open_modes, seed=9, reps=R, m=m)
    y, _ = oracle.m1_estimate(X, edges, open_modes, m=m, bins=bins, signs=signs)
    for o in range(2):
        Xs = [X[0], X[1][:, :, o], X[2]]
        edges_s = [(1, 2), (3, 4), (5, 0)]
        ys, _ = oracle.m1_estimate(Xs, edges_s, [], m=m, bins=bins, signs=signs)
        assert np.allclose(y[:, o], ys[:, 0], rtol=1e-12, atol=1e-12)


def test_unbiased_and_within_variance_bound_on_cyclic_network():
    # Lemma "general-expectation-variance": E[y] = tc, Var(y) <= 3^t/m prod ||X_k||^2
    rng = np.random.default_rng(7)
    X = [rng.standard_normal((4, 4)) for _ in range(3)]
    edges = [(1, 2), (3, 4), (5, 0)]
    m, R = 8, 20000
    y, _ = oracle.m1_estimate(X, edges, [], m=m, reps=R, seed=21)
    y = y[:, 0]
    tc = oracle.tc_einsum(X, edges, [])
    assert abs(y.mean() - tc) <= 5 * y.std() / np.sqrt(R)
    bound = 3 ** len(edges) / m * oracle.frobenius_product(X) ** 2
    assert y.var() <= bound * (1 + 5 * np.sqrt(2 / R))


def test_scalar_and_empty_tensors():
    # a scalar network and a contraction over an empty mode
    y, _ = oracle.m1_estimate([np.array(3.0), np.array(-2.0)], [], [], m=4, reps=2, seed=1)
    assert np.allclose(y, -6.0)
    y, _ = oracle.m1_estimate([np.zeros((0, 3)), np.zeros((0,))], [(0, 2)], [1], m=4, reps=2, seed=1)
    assert np.allclose(y, 0.0) and y.shape == (2, 3)
