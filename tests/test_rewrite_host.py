"""The library's WLOG rewrites (Sec. 4.1) on the host, through the C ABI
(tnsk_rewrite, no GPU needed): the network it plans for random networks with
hyperedges (method 1: copy tensors) and with traces / repeated contractions
(method 2: diagonal sums and reshapes) has the shapes, contractions and copy flags
of the oracle's own rewrite (oracle/normalize.py), which the oracle pins tie to tc."""
import numpy as np
import pytest

from oracle.normalize import copy_tensors, needs_normalize, normalize

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def tnsk():
    from paper_2603_07387_gb300 import build, tnsk as t

    build.build()
    return t


def _random_network(rng, hyper):
    p = int(rng.integers(1, 5))
    orders = [int(rng.integers(0, 5)) for _ in range(p)]
    q = sum(orders)
    modes = list(rng.permutation(q))
    edges = []
    while len(modes) >= 2 and rng.random() < 0.8:
        edges.append((int(modes.pop()), int(modes.pop())))
        if hyper and modes and rng.random() < 0.4:  # a second contraction on an existing mode
            edges.append((edges[int(rng.integers(0, len(edges)))][0], int(modes.pop())))
    parent = list(range(q))

    def find(a):
        while parent[a] != a:
            a = parent[a]
        return a

    for u, v in edges:
        parent[find(u)] = find(v)
    dims = [int(rng.integers(1, 4)) for _ in range(q)]
    dims = [dims[find(g)] for g in range(q)]  # equal dims within a class
    shapes, g = [], 0
    for k in range(p):
        shapes.append(tuple(dims[g:g + orders[k]]))
        g += orders[k]
    return shapes, edges


@pytest.mark.parametrize("hyper", [True, False])
def test_rewrite_matches_the_oracle_on_random_networks(tnsk, hyper):
    rng = np.random.default_rng(7 if hyper else 8)
    method = tnsk.GENERAL if hyper else tnsk.ACYCLIC
    for _ in range(400):
        shapes, edges = _random_network(rng, hyper)
        net = tnsk.Network([torch.zeros(s) for s in shapes], edges, [])
        got = tnsk.rewrite(net, tnsk.Params(m=8, reps=1, method=method))
        X = [np.zeros(s) for s in shapes]
        if hyper:
            T, E, _ = copy_tensors(X, edges)
            copy = [False] * len(shapes) + [True] * (len(T) - len(shapes))
        elif needs_normalize(X, edges):
            T, E, _ = normalize(X, edges)
            copy = [False] * len(T)
        else:
            T, E, copy = X, list(edges), [False] * len(X)
        assert got == ([t.shape for t in T], E, copy), (shapes, edges)


def test_rewrite_of_the_paper_examples_and_its_errors(tnsk):
    # WLOG 1: b's mode in two contractions -> one order-3 copy tensor
    vs = [torch.zeros(5) for _ in range(3)]
    got = tnsk.rewrite(tnsk.Network(vs, [(0, 1), (1, 2)], []), tnsk.Params(m=8, reps=1))
    assert got == ([(5,), (5,), (5,), (5, 5, 5)], [(0, 3), (1, 4), (2, 5)], [False, False, False, True])
    # WLOG 3: two matrices joined twice -> vec(A) . vec(B)
    AB = [torch.zeros(3, 4), torch.zeros(3, 4)]
    got = tnsk.rewrite(tnsk.Network(AB, [(0, 2), (1, 3)], []), tnsk.Params(m=8, reps=1, method=tnsk.ACYCLIC))
    assert got == ([(12,), (12,)], [(0, 1)], [False, False])
    # WLOG 2: a full trace leaves an order-0 tensor
    got = tnsk.rewrite(tnsk.Network([torch.zeros(4, 4)], [(1, 0)], []),
                       tnsk.Params(m=8, reps=1, method=tnsk.ACYCLIC))
    assert got == ([()], [], [False])
    # a class of 13 modes: beyond the copy tensor's order limit
    vs = [torch.zeros(2) for _ in range(13)]
    with pytest.raises(tnsk.TnskError) as e:
        tnsk.rewrite(tnsk.Network(vs, [(0, k) for k in range(1, 13)], []), tnsk.Params(m=8, reps=1))
    assert e.value.status == -3
    # a grouped tensor that would need a trace
    a = torch.zeros(2, 3, 2)
    with pytest.raises(tnsk.TnskError) as e:
        tnsk.rewrite(tnsk.Network([tnsk.Rung(a, a)], [(0, 1)], []), tnsk.Params(m=8, reps=1, method=tnsk.ACYCLIC))
    assert e.value.status == -3
