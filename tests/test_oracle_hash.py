"""Oracle pins for the hash contract (count sketch, Sec. 2.1 Def. "Count sketch").

The paper only requires 2-wise independent bins and 4-wise independent signs
(Def. "k-wise independence"); the contract's generator is SplitMix64, pinned to
its published reference outputs, and the families are checked statistically."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1
P61 = (1 << 61) - 1


def test_splitmix64_reference_sequence():
    rows = []
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            s, o = line.split()
            rows.append((int(s, 16), int(o, 16)))
    assert len(rows) == 3
    for state, out in rows:
        assert oracle.splitmix64(state) == out


def _py_hash(seed, rep, tid, n, m):
    """The contract evaluated with Python integers (exact, no 128-bit tricks)."""
    sm = oracle.splitmix64
    key = sm(sm(sm(seed) ^ rep) ^ tid)

    def red(x):
        return x % P61

    a0, a1 = red(sm(key ^ 0)), red(sm(key ^ 1))
    c = [red(sm(key ^ (8 + j))) for j in range(4)]
    bins = [((a1 * i + a0) % P61) % m for i in range(n)]
    signs = [(-1 if ((c[3] * i**3 + c[2] * i**2 + c[1] * i + c[0]) % P61) & 1 else 1) for i in range(n)]
    return np.array(bins), np.array(signs)


@pytest.mark.parametrize("seed,rep,tid,n,m", [(0, 0, 1 << 56, 50, 16), (0x7E57, 5, (4 << 56) | 12345, 300, 1024),
                                              (2**63 + 11, 63, 2 << 56, 17, 1), (3, 1, 7, 40, 65536)])
def test_count_sketch_matches_big_integer_evaluation(seed, rep, tid, n, m):
    b, s = oracle.count_sketch(seed, rep, tid, n, m)
    pb, ps = _py_hash(seed, rep, tid, n, m)
    assert np.array_equal(b, pb)
    assert np.array_equal(s, ps)


def test_large_index_values_reduce_mod_p():
    # indices beyond 2^31 are legal domain values; the 128-bit mulmod must agree
    b, s = oracle.count_sketch(9, 0, 1, 5, 256)
    assert b.min() >= 0 and b.max() < 256 and set(np.unique(s)) <= {-1, 1}


def test_bins_uniform_and_pairwise_independent():
    m, n, reps = 16, 8, 4000
    B = np.stack([oracle.count_sketch(11, r, 1 << 56, n, m)[0] for r in range(reps)])
    # marginal uniformity: chi-square over all (index, bin) cells
    cnt = np.stack([np.bincount(B[:, i], minlength=m) for i in range(n)])
    exp = reps / m
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    dof = n * (m - 1)
    assert chi2 < dof + 6 * np.sqrt(2 * dof)
    # 2-wise: collision probability of distinct items is 1/m
    coll = np.mean([np.mean(B[:, i] == B[:, j]) for i in range(n) for j in range(i + 1, n)])
    assert abs(coll - 1 / m) < 5 * np.sqrt((1 / m) / (reps * n * (n - 1) / 2)) + 0.005


def test_signs_four_wise_moments_vanish():
    n, reps = 6, 20000
    S = np.stack([oracle.count_sketch(12, r, 2 << 56, n, 8)[1] for r in range(reps)]).astype(np.float64)
    tol = 5 / np.sqrt(reps)
    assert np.all(np.abs(S.mean(0)) < tol)
    for a in range(n):
        for b in range(a + 1, n):
            assert abs(np.mean(S[:, a] * S[:, b])) < tol
    for quad in [(0, 1, 2, 3), (1, 2, 4, 5), (0, 2, 3, 5)]:
        assert abs(np.mean(np.prod(S[:, list(quad)], axis=1))) < tol


def test_tables_are_deterministic_and_keyed():
    a = oracle.count_sketch(1, 2, 3, 100, 64)
    b = oracle.count_sketch(1, 2, 3, 100, 64)
    c = oracle.count_sketch(1, 3, 3, 100, 64)
    d = oracle.count_sketch(1, 2, 4, 100, 64)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0]) and not np.array_equal(a[0], d[0])


def test_table_ids_are_distinct_per_role():
    ids = {oracle.tid(1, 5), oracle.tid(2, 5), oracle.tid(3, 5, 1), oracle.tid(4, 5, 1, 0, 0), oracle.tid(4, 5, 1, 0, 1),
           oracle.tid(4, 5, 2, 0, 0)}
    assert len(ids) == 6
