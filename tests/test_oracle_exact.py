"""Oracle pins for the exact contraction (Def. "Tensor contraction", Def. "TNC")."""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ex(name):
    with open(os.path.join(GOLDEN, "paper_examples.json")) as f:
        return json.load(f)[name]


def test_example1_reduced_form():
    ex = _ex("example1")
    rng = np.random.default_rng(1)
    dims = {1: 3, 2: 2, 3: 2, 4: 2, 5: 3, 6: 2, 7: 2, 8: 3}  # n_u = n_v on every edge
    shapes, g = [], 1
    for q in ex["orders"]:
        shapes.append(tuple(dims[g + j] for j in range(q)))
        g += q
    X = [rng.standard_normal(s) for s in shapes]
    edges = [(u - 1, v - 1) for u, v in ex["edges"]]
    K = sorted({m for e in ex["edges"] for m in e})
    assert K == ex["K"]
    open_modes = [g - 1 for g in ex["K_open"]]
    want = np.einsum(ex["reduced_einsum"], *X)
    assert np.allclose(oracle.tc_definition(X, edges, open_modes), want)
    assert np.allclose(oracle.tc_reduced(X, edges, open_modes), want)
    assert np.allclose(oracle.tc_einsum(X, edges, open_modes), want)


def test_closed_forms():
    rng = np.random.default_rng(2)
    A, B, C = (rng.standard_normal((4, 4)) for _ in range(3))
    # tr(ABC): modes A=(0,1), B=(2,3), C=(4,5)
    tri = [(1, 2), (3, 4), (5, 0)]
    want = np.trace(A @ B @ C)
    assert np.isclose(oracle.tc_definition([A, B, C], tri, []), want)
    assert np.isclose(oracle.tc_einsum([A, B, C], tri, []), want)
    # AB = tc(A x B, {(2,3)}) (footnote to the ATNC paragraph, 1-based)
    assert np.allclose(oracle.tc_definition([A, B], [(1, 2)], [0, 3]), A @ B)
    assert np.allclose(oracle.tc_definition([A, B], [(1, 2)], [3, 0]), (A @ B).T)
    # inner product and trace (a contraction inside one tensor)
    x, y = rng.standard_normal(5), rng.standard_normal(5)
    assert np.isclose(oracle.tc_reduced([x, y], [(0, 1)], []), x @ y)
    assert np.isclose(oracle.tc_definition([A], [(0, 1)], []), np.trace(A))
    # a scalar network
    assert np.isclose(oracle.tc_definition([np.array(2.5)], [], []), 2.5)


def test_triangle_count_corollary():
    ex = _ex("triangle")
    rng = np.random.default_rng(3)
    n = 6
    A = (rng.random((n, n)) < 0.5).astype(float)
    A = np.triu(A, 1)
    A = A + A.T
    edges = [(u - 1, v - 1) for u, v in ex["edges"]]
    tc = oracle.tc_einsum([A, A, A], edges, [])
    # undirected simple graph: tr(A^3) = 6 x number of triangles
    tri = sum(A[i, j] * A[j, k] * A[k, i] for i in range(n) for j in range(i + 1, n) for k in range(j + 1, n))
    assert np.isclose(tc, 6 * tri)
    assert np.isclose(oracle.tc_reduced([A, A, A], edges, []), np.trace(A @ A @ A))


@pytest.mark.parametrize("seed", range(4))
def test_three_exact_forms_agree_on_random_networks(seed):
    rng = np.random.default_rng(100 + seed)
    # random small network with a cycle, a self-contraction and open legs
    X = [rng.standard_normal((2, 3, 2)), rng.standard_normal((3, 2)), rng.standard_normal((2, 2, 2))]
    # modes: X0=(0,1,2) X1=(3,4) X2=(5,6,7)
    edges = [(1, 3), (4, 5), (2, 6)]
    open_modes = [7, 0]
    a = oracle.tc_definition(X, edges, open_modes)
    b = oracle.tc_reduced(X, edges, open_modes)
    c = oracle.tc_einsum(X, edges, open_modes)
    assert np.allclose(a, b) and np.allclose(a, c)
    # self contraction inside X2: modes 5 and 7
    edges2 = [(1, 3), (4, 6), (5, 7)]
    a = oracle.tc_definition(X, edges2, [0, 2])
    c = oracle.tc_einsum(X, edges2, [0, 2])
    assert np.allclose(a, c)
    assert np.allclose(a, oracle.tc_sequential(X, edges2, [0, 2]))
    assert np.allclose(oracle.tc_definition(X, edges, open_modes), oracle.tc_sequential(X, edges, open_modes))


def test_sequential_contraction_on_grids_and_the_triangle():
    from paper_2603_07387_gb300 import workloads as W

    for L1, L2, b in [(1, 3, 3), (2, 2, 3), (2, 3, 2), (3, 3, 2)]:
        g = W.grid(L1, L2, b, seed=L1 * 10 + L2)
        want = oracle.tc_definition(g.tensors, g.edges, g.open) if L1 * L2 <= 6 else oracle.tc_einsum(
            g.tensors, g.edges, g.open)
        assert np.allclose(oracle.tc_sequential(g.tensors, g.edges, g.open), want, rtol=1e-12)
    rng = np.random.default_rng(5)
    A, B, C = rng.standard_normal((4, 5)), rng.standard_normal((5, 6)), rng.standard_normal((6, 4))
    assert np.isclose(oracle.tc_sequential([A, B, C], [(1, 2), (3, 4), (5, 0)], []), np.trace(A @ B @ C))
    # an open leg kept in the requested order
    out = oracle.tc_sequential([A, B], [(1, 2)], [3, 0])
    assert np.allclose(out, (A @ B).T)


def test_frobenius_product():
    x = [np.ones((2, 2)), 2 * np.ones(3)]
    assert np.isclose(oracle.frobenius_product(x), 2.0 * np.sqrt(12))
