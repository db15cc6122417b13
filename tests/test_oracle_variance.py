"""Pins the exact variance of the all-ones chain (oracle/variance.py, the estimator of
Lemma "exponential-dependence") by brute force: the mean and variance of y = ||s||^2
over every choice of bin and sign functions on tiny domains, all equally likely (fully
random functions are k-wise independent for every k), with s the tensor sketch of the
all-ones order-q tensor computed straight from its definition."""
import itertools

import numpy as np
import pytest

from oracle.variance import chain_allones_variance, lemma_lower_bound


def _brute(n, q, m):
    idx = list(itertools.product(range(n), repeat=q))
    bins_all = list(itertools.product(range(m), repeat=n))
    signs_all = list(itertools.product((1, -1), repeat=n))
    per_mode = [(h, s) for h in bins_all for s in signs_all]
    ys = []
    for funcs in itertools.product(per_mode, repeat=q):
        sk = np.zeros(m)
        for i in idx:
            b = sum(funcs[k][0][i[k]] for k in range(q)) % m
            sg = 1
            for k in range(q):
                sg *= funcs[k][1][i[k]]
            sk[b] += sg
        ys.append(float(np.dot(sk, sk)))
    ys = np.array(ys)
    return ys.mean(), ys.var()


@pytest.mark.parametrize("n,q,m", [(2, 2, 2), (2, 2, 3), (2, 2, 4), (3, 2, 2), (2, 3, 2), (2, 3, 4), (3, 2, 3)])
def test_exact_variance_matches_enumeration(n, q, m):
    mean, var = _brute(n, q, m)
    assert mean == pytest.approx(n ** q, rel=1e-12)  # unbiased: E[y] = tc = n^q
    assert var / n ** (2 * q) == pytest.approx(chain_allones_variance(n, q, m), rel=1e-12)


def test_large_n_limit_and_the_lemma():
    # n -> infinity: 2 (2^q - 1) / m + 2 (3^q - 2^{q+1} + 1) / m^2 for even m
    q, m = 10, 64
    lim = 2 * (2 ** q - 1) / m + 2 * (3 ** q - 2 ** (q + 1) + 1) / m ** 2
    assert chain_allones_variance(10 ** 9, q, m) == pytest.approx(lim, rel=1e-6)
    # the lemma's lower bound holds in that limit (leading 3^q / m^2 coefficient 2 > 1/2)
    for q in (2, 4, 8, 16, 24):
        assert chain_allones_variance(10 ** 9, q, 256) >= lemma_lower_bound(q, 256)
    # but not for every n: at n = 8, m = 256 the exact variance falls below the stated
    # bound from q = 20 on ((3 - 2/n)^q grows slower than 3^q)
    assert chain_allones_variance(8, 16, 256) >= lemma_lower_bound(16, 256)
    assert chain_allones_variance(8, 20, 256) < lemma_lower_bound(20, 256)
