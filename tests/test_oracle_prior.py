"""Oracle pins for the earlier cross-correlation estimator (the prior method of
Sec. 4.2, its two examples): it reduces to the textbook count-sketch inner product
for one contraction, equals method 1 with the conjugated tensor's modes taking the
complement on the acyclic example x - Y - z, matches the example's Fourier formula
e_1^T F^-1(F x_1 o conj(F x_2) o F x_3) written as a bin-sum condition, and on the
cyclic example its mean over seeds approaches P(2h = 0 mod m) tc, not tc."""
import numpy as np
import pytest

import oracle
from oracle import prior


def test_one_contraction_is_the_count_sketch_inner_product():
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(50), rng.standard_normal(50)
    m, seed = 16, 3
    est = prior.estimate([x, y], [(0, 1)], [], m, 4, seed)
    for r in range(4):
        b, s = oracle.count_sketch(seed, r, oracle.tid(1, 0), 50, m)
        cx, cy = np.zeros(m), np.zeros(m)
        np.add.at(cx, b, s * x)
        np.add.at(cy, b, s * y)
        assert np.isclose(est[r, 0], cx @ cy)


def test_acyclic_example_equals_method1_with_the_middle_tensor_complemented():
    """x (mode 0), Y (modes 1, 2), z (mode 3): the chain conjugates Y, which method 1
    expresses by giving Y's modes the complement (edge (u, v): v takes C')."""
    rng = np.random.default_rng(2)
    x, Y, z = rng.standard_normal(7), rng.standard_normal((7, 5)), rng.standard_normal(5)
    m, seed, R = 32, 11, 6
    got = prior.estimate([x, Y, z], [(0, 1), (2, 3)], [], m, R, seed)
    want, _ = oracle.m1_estimate([x, Y, z], [(0, 1), (3, 2)], [], m=m, reps=R, seed=seed)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)


def test_cyclic_example_matches_the_fourier_formula():
    """tr-like network X(1,2) Y(3,4) Z(5,6) with (2,3), (4,5), (1,6) (1-based): the
    estimate is sum over bins b1 - b2 + b3 = 0 (mod m) of x_1(b1) x_2(b2) x_3(b3),
    the Fourier formula of the example with the middle spectrum conjugated."""
    rng = np.random.default_rng(3)
    X, Y, Z = (rng.standard_normal((4, 4)) for _ in range(3))
    edges = [(1, 2), (3, 4), (5, 0)]
    m, seed = 8, 5
    got = prior.estimate([X, Y, Z], edges, [], m, 3, seed)
    for r in range(3):
        tabs = [oracle.count_sketch(seed, r, oracle.tid(1, e), 4, m) for e in range(3)]
        (h1, s1), (h2, s2), (h3, s3) = tabs
        sx, sy, sz = np.zeros(m), np.zeros(m), np.zeros(m)
        for i in range(4):
            for j in range(4):
                sx[(h3[i] + h1[j]) % m] += s3[i] * s1[j] * X[i, j]   # X: modes 1 (edge 3), 2 (edge 1)
                sy[(h1[i] + h2[j]) % m] += s1[i] * s2[j] * Y[i, j]
                sz[(h2[i] + h3[j]) % m] += s2[i] * s3[j] * Z[i, j]
        want = sum(sx[a] * sy[b] * sz[c] for a in range(m) for b in range(m) for c in range(m)
                   if (a - b + c) % m == 0)
        assert np.isclose(got[r, 0], want)


def test_cyclic_example_is_biased():
    """Mean over many seeds on the triangle: about tc * P(2h = 0 mod m) (the edge
    (1, 6) joins two unconjugated tensors), while method 1 is unbiased."""
    rng = np.random.default_rng(4)
    X, Y, Z = (rng.uniform(0, 1, (3, 3)) for _ in range(3))
    edges = [(1, 2), (3, 4), (5, 0)]
    tc = np.trace(X @ Y @ Z)
    m, S = 8, 1500
    ys = np.concatenate([prior.estimate([X, Y, Z], edges, [], m, 50, seed)[:, 0] for seed in range(S // 50)])
    # P(2 h(i) = 0 mod m) over the seeds, measured on the same hash family
    hit = np.mean([(2 * oracle.count_sketch(seed, r, oracle.tid(1, 2), 3, m)[0] % m == 0).mean()
                   for seed in range(S // 50) for r in range(50)])
    se = ys.std(ddof=1) / np.sqrt(ys.size)
    assert abs(ys.mean() - hit * tc) <= 5 * se
    assert abs(hit - 2 / m) < 0.05
    assert abs(ys.mean() - tc) > 10 * se  # far from tc: the prior method fails on the cycle
    y1, _ = oracle.m1_estimate([X, Y, Z], edges, [], m=m, reps=S, seed=1)
    assert abs(y1.mean() - tc) <= 5 * y1.std(ddof=1) / np.sqrt(S)


@pytest.mark.parametrize("open_modes", [[0, 3], [3, 0]])
def test_open_legs_per_output_entry(open_modes):
    """With open legs each output entry is the estimator on the sub-network at that
    open index (Corollary "full-to-partial-tc"), in the order of the open list."""
    rng = np.random.default_rng(5)
    A, B = rng.standard_normal((3, 6)), rng.standard_normal((6, 2))  # modes 0,1 / 2,3
    m, seed = 16, 9
    got = prior.estimate([A, B], [(1, 2)], open_modes, m, 2, seed)
    dims = {0: 3, 3: 2}
    for o, idx in enumerate(np.ndindex(*[dims[g] for g in open_modes])):
        at = dict(zip(open_modes, idx))
        want = prior.estimate([A[at[0]], B[:, at[3]]], [(0, 1)], [], m, 2, seed)[:, 0]
        assert np.allclose(got[:, o], want)


def test_even_ring_is_unbiased():
    """A ring of four matrices: the chain conjugates tensors 0 and 2, so every
    contraction joins a conjugated and an unconjugated tensor and the mean over seeds
    approaches tc (the odd ring above does not)."""
    rng = np.random.default_rng(9)
    Ms = [rng.uniform(0, 1, (3, 3)) for _ in range(4)]
    edges = [(1, 2), (3, 4), (5, 6), (7, 0)]
    tc = np.trace(Ms[0] @ Ms[1] @ Ms[2] @ Ms[3])
    ys = np.concatenate([prior.estimate(Ms, edges, [], 8, 50, seed)[:, 0] for seed in range(30)])
    se = ys.std(ddof=1) / np.sqrt(ys.size)
    assert abs(ys.mean() - tc) <= 5 * se
