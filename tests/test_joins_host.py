"""Host layout of join-size estimation (Sec. 5.1, Corollary "multi-join-card-est"):
the frequency tensors and equi-join contractions that joins.join_network lays out,
with the hyperedge of a three-way class turned into a copy tensor (the oracle's
WLOG 1 rewrite, the same order the library uses), contract exactly to COUNT(*) of
the join computed by brute force over the tuples."""
import itertools

import numpy as np

import oracle
from oracle.normalize import copy_tensors
from paper_2603_07387_gb300 import joins


def _count(relations, equalities):
    n = 0
    for combo in itertools.product(*[range(len(r)) for r in relations]):
        if all(relations[k1][combo[k1]][c1] == relations[k2][combo[k2]][c2] for (k1, c1), (k2, c2) in equalities):
            n += 1
    return n


def test_paper_query_layout_counts_the_join():
    rng = np.random.default_rng(3)
    R1 = rng.integers(0, 4, (7, 1))
    R2 = np.stack([rng.integers(0, 4, 9), rng.integers(0, 3, 9)], 1)
    R3 = rng.integers(0, 4, (6, 1))
    R4 = rng.integers(0, 3, (5, 1))
    eq = [((0, 0), (1, 0)), ((2, 0), (1, 0)), ((3, 0), (1, 1))]
    jn = joins.join_network([R1, R2, R3, R4], eq)
    assert [len(s) for s in jn.shapes] == [1, 2, 1, 1] and len(jn.edges) == 3
    X, E, _ = copy_tensors(joins.exact_dense_tensors(jn), jn.edges)
    assert float(oracle.tc_definition(X, E, [])) == _count([R1, R2, R3, R4], eq)


def test_two_way_joins_and_unjoined_columns():
    """A chain R1.0 = R2.0, R2.1 = R3.1 with columns that join nothing (summed out)."""
    rng = np.random.default_rng(4)
    R1 = rng.integers(0, 3, (6, 2))
    R2 = rng.integers(0, 3, (8, 2))
    R3 = rng.integers(0, 3, (5, 3))
    eq = [((0, 0), (1, 0)), ((1, 1), (2, 1))]
    jn = joins.join_network([R1, R2, R3], eq)
    assert [len(s) for s in jn.shapes] == [1, 2, 1]
    X = joins.exact_dense_tensors(jn)
    assert float(oracle.tc_definition(X, jn.edges, [])) == _count([R1, R2, R3], eq)
    assert sum(len(u) for u in jn.updates) == len(R1) + len(R2) + len(R3)
