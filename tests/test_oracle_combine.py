"""Oracle pins for the combination of repetitions (Theorem 1: median trick)."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("R,g", [(12, 1), (12, 3), (12, 4), (12, 12), (7, 7), (1, 1)])
def test_median_of_group_means(R, g):
    rng = np.random.default_rng(R * 10 + g)
    a = rng.standard_normal((R, 5))
    got = oracle.combine(a, g)
    means = a.reshape(g, R // g, 5).mean(axis=1)
    assert np.allclose(got, np.median(means, axis=0), rtol=1e-15, atol=1e-15)


def test_median_is_robust_to_an_outlier_group():
    a = np.array([1.0, 1.1, 0.9, 1e9, 1.0, 0.95])
    assert np.isclose(oracle.combine(a, 6)[0], 1.0)
    assert oracle.combine(a, 1)[0] > 1e8


def test_rejects_uneven_groups():
    with pytest.raises(oracle.OracleError):
        oracle.combine(np.zeros((10, 1)), 3)
