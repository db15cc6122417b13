"""Oracle pins for the WLOG 2 / WLOG 3 rewrite (Sec. 4.1) the acyclic method needs.

The rewrite must keep tc (checked against the literal definition by brute force),
reduce to the paper's examples (tr, vec(A) . vec(B)) and follow the stated mode
order (checked on hand-worked cases)."""
import numpy as np
import pytest

import oracle
from oracle.normalize import needs_normalize, normalize


def test_wlog3_example_is_the_vec_inner_product():
    """Two matrices joined on both modes become vec(A), vec(B) and one contraction."""
    rng = np.random.default_rng(3)
    A, B = rng.standard_normal((3, 4)), rng.standard_normal((3, 4))
    T, E, O = normalize([A, B], [(0, 2), (1, 3)])
    assert E == [(0, 1)] and O == []
    assert np.array_equal(T[0], A.reshape(-1)) and np.array_equal(T[1], B.reshape(-1))
    assert np.isclose(oracle.tc_definition(T, E, []), np.sum(A * B))


def test_wlog3_group_order_follows_the_edge_list():
    """Edges listed (1,3) before (0,2): the merged index is i_1 * n_0 + i_0, so A
    and B are both transposed before vec."""
    rng = np.random.default_rng(4)
    A, B = rng.standard_normal((3, 4)), rng.standard_normal((3, 4))
    T, E, _ = normalize([A, B], [(1, 3), (0, 2)])
    assert E == [(0, 1)]
    assert np.array_equal(T[0], A.T.reshape(-1)) and np.array_equal(T[1], B.T.reshape(-1))


def test_wlog2_trace_of_a_matrix_and_a_partial_trace():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((4, 3, 4))  # modes 0, 1, 2; (0, 2) traced
    v = rng.standard_normal(3)          # mode 3
    T, E, O = normalize([A, v], [(0, 2), (1, 3)])
    want = sum(A[i, :, i] for i in range(4))
    assert np.allclose(T[0], want) and T[0].shape == (3,)
    assert np.array_equal(T[1], v) and E == [(0, 1)] and O == []
    M = rng.standard_normal((5, 5))
    T, E, _ = normalize([M], [(1, 0)])
    assert T[0].shape == () and np.isclose(T[0], np.trace(M)) and E == []


def test_mode_positions_and_renumbering():
    """X (modes 0..3) joins Y on its modes 3 and 1 (edges in that order) and is open
    on 0 and 2: X' = [open 0, merged (3, 1), open 2]; the merged mode stands where
    the group's lowest mode (1) was."""
    rng = np.random.default_rng(6)
    X = rng.standard_normal((2, 3, 5, 4))
    Y = rng.standard_normal((4, 3, 6))  # modes 4, 5, 6
    edges = [(3, 4), (1, 5)]
    T, E, O = normalize([X, Y], edges, open_modes=[2, 0, 6])
    assert T[0].shape == (2, 12, 5) and T[1].shape == (12, 6)
    assert np.array_equal(T[0], X.transpose(0, 3, 1, 2).reshape(2, 12, 5))
    assert np.array_equal(T[1], Y.reshape(12, 6))
    assert E == [(1, 3)] and O == [2, 0, 4]
    want = oracle.tc_definition([X, Y], edges, [2, 0, 6])
    assert np.allclose(oracle.tc_definition(T, E, O), want)


def test_flipped_orientations_within_a_group():
    """e_1 = (X, Y), e_2 = (Y, X): the merged contraction keeps e_1's orientation."""
    rng = np.random.default_rng(7)
    X, Y = rng.standard_normal((2, 3)), rng.standard_normal((3, 2))  # modes 0,1 / 2,3
    T, E, _ = normalize([X, Y], [(0, 3), (2, 1)])
    assert E == [(0, 1)]
    assert np.array_equal(T[0], X.reshape(-1)) and np.array_equal(T[1], Y.T.reshape(-1))
    assert np.isclose(oracle.tc_definition(T, E, []), np.sum(X * Y.T))


@pytest.mark.parametrize("seed", range(8))
def test_random_networks_keep_tc(seed):
    """Random small networks with traces, double and triple contractions between
    pairs: tc before == tc after (brute-force definition), and the result needs no
    further rewrite."""
    rng = np.random.default_rng(100 + seed)
    p = int(rng.integers(2, 4))
    orders = [int(rng.integers(2, 5)) for _ in range(p)]
    q = sum(orders)
    modes = list(rng.permutation(q))
    edges = []
    while len(modes) >= 2 and len(edges) < q // 2:
        u, v = int(modes.pop()), int(modes.pop())
        edges.append((u, v))
    dims = [int(rng.integers(1, 4)) for _ in range(q)]
    for u, v in edges:
        dims[v] = dims[u]
    tensors, g = [], 0
    for k in range(p):
        tensors.append(rng.standard_normal(tuple(dims[g:g + orders[k]])))
        g += orders[k]
    open_modes = [int(x) for x in rng.permutation([g for g in range(q) if all(g not in e for e in edges)])]
    T, E, O = normalize(tensors, edges, open_modes)
    assert not needs_normalize(T, E)
    want = oracle.tc_definition(tensors, edges, open_modes)
    assert np.allclose(oracle.tc_definition(T, E, O), want, atol=1e-10)


def test_needs_normalize():
    A, B, C = np.ones((2, 2)), np.ones((2, 2)), np.ones((2, 2))
    assert not needs_normalize([A, B, C], [(1, 2), (3, 4)])
    assert needs_normalize([A, B, C], [(0, 1)])                 # trace
    assert needs_normalize([A, B, C], [(0, 2), (1, 3)])         # double contraction


def test_wlog1_paper_example_and_copy_tensor_layout():
    """a, b, c vectors with b's mode in two contractions: sum_i a(i) b(i) c(i); the
    rewrite appends one order-3 copy tensor joined to modes 0, 1, 2 in order."""
    from oracle.normalize import copy_tensors
    rng = np.random.default_rng(8)
    a, b, c = (rng.standard_normal(5) for _ in range(3))
    T, E, O = copy_tensors([a, b, c], [(0, 1), (1, 2)])
    assert len(T) == 4 and T[3].shape == (5, 5, 5) and E == [(0, 3), (1, 4), (2, 5)] and O == []
    assert T[3].sum() == 5 and all(T[3][i, i, i] == 1 for i in range(5))
    assert np.isclose(oracle.tc_definition(T, E, []), np.sum(a * b * c))
    assert np.isclose(oracle.tc_definition([a, b, c], [(0, 1), (1, 2)], []), np.sum(a * b * c))


@pytest.mark.parametrize("seed", range(6))
def test_wlog1_random_hyperedges_keep_tc(seed):
    """Random networks where modes join two or three contractions (classes of 3-4 modes,
    repeated pairs, two-mode classes mixed in, open modes): tc (brute-force definition,
    which reads every bracket) is unchanged and no mode is left in two contractions."""
    from oracle.normalize import copy_tensors
    rng = np.random.default_rng(300 + seed)
    shapes = [(2, 3), (3, 2), (3,), (2, 2)]
    tensors = [rng.standard_normal(s) for s in shapes]  # modes 0,1 | 2,3 | 4 | 5,6
    dims = [2, 3, 3, 2, 3, 2, 2]
    classes = [[1, 2, 4], [0, 3, 5]] if seed % 2 else [[1, 2, 4], [0, 5]]
    edges = []
    for cl in classes:
        order = list(rng.permutation(cl))
        edges += [(int(order[i]), int(order[i + 1])) for i in range(len(order) - 1)]
        if len(cl) >= 3 and seed % 3 == 0:
            edges.append((int(order[-1]), int(order[0])))  # a redundant cycle of brackets
    if seed % 2 == 0:
        edges.append(edges[-1])  # a repeated pair
    assert all(dims[u] == dims[v] for u, v in edges)
    open_modes = [g for g in range(7) if all(g not in e for e in edges)]
    T, E, O = copy_tensors(tensors, edges, open_modes)
    used = [g for e in E for g in e]
    assert len(used) == len(set(used))
    want = oracle.tc_definition(tensors, edges, open_modes)
    assert np.allclose(oracle.tc_definition(T, E, O), want)


def test_method2_on_the_rewrite_estimates_the_original():
    """Method 2 on the rewritten network (a trace and a double contraction removed) is
    unbiased for the original network's tc: mean over many reps within 5 standard
    errors."""
    rng = np.random.default_rng(12)
    A = rng.uniform(0, 1, (3, 2, 4, 4))  # modes 0-3: (2, 3) traced
    B = rng.uniform(0, 1, (2, 3, 5))     # modes 4-6: joins A twice
    C = rng.uniform(0, 1, (5,))          # mode 7
    edges = [(1, 4), (0, 5), (2, 3), (6, 7)]
    tc = float(oracle.tc_definition([A, B, C], edges, []))
    T, E, _ = normalize([A, B, C], edges)
    y, _ = oracle.m2_estimate(T, E, m=16, reps=4000, seed=3, root=2)
    se = y.std(ddof=1) / np.sqrt(y.size)
    assert abs(y.mean() - tc) <= 5 * se


def test_method1_on_copy_tensors_estimates_the_hyperedge_network():
    """Method 1 on the WLOG 1 rewrite (one copy tensor of order 3) is unbiased for the
    original network's tc (the brute-force definition reads the hyperedge's brackets)."""
    from oracle.normalize import copy_tensors
    rng = np.random.default_rng(13)
    X = [rng.uniform(0, 1, (4, 3)), rng.uniform(0, 1, (3, 4)), rng.uniform(0, 1, (4,))]  # modes 0,1 | 2,3 | 4
    edges = [(0, 3), (3, 4), (1, 2)]  # mode 3 in two contractions: class {0, 3, 4}
    tc = float(oracle.tc_definition(X, edges, []))
    T, E, _ = copy_tensors(X, edges)
    y, _ = oracle.m1_estimate(T, E, [], m=16, reps=4000, seed=4)
    se = y.std(ddof=1) / np.sqrt(y.size)
    assert abs(y.mean() - tc) <= 5 * se
