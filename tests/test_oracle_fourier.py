"""Oracle pins for the transform (Sec. 2: DFT matrix F, Lemma "conv-thm")."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("m", [1, 2, 4, 8, 64, 256])
def test_fft_equals_dft_definition_and_numpy(m):
    rng = np.random.default_rng(m)
    x = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    a = oracle.fft(x)
    b = oracle.dft(x)
    assert np.allclose(a, b, rtol=0, atol=1e-10 * max(1, np.abs(x).sum()))
    assert np.allclose(a, np.fft.fft(x), rtol=0, atol=1e-10 * max(1, np.abs(x).sum()))


def test_dft_closed_forms():
    m = 16
    d = np.zeros(m)
    d[0] = 1
    assert np.allclose(oracle.fft(d), np.ones(m))  # F e_1 = 1
    assert np.allclose(oracle.fft(np.ones(m)), m * d)  # F 1 = m e_1
    k = 3
    e = np.zeros(m)
    e[k] = 1  # F e_{k+1} = exp(-2 pi i j k / m)
    assert np.allclose(oracle.fft(e), np.exp(-2j * np.pi * np.arange(m) * k / m))


def _circ_conv(x, y):
    # Def. "Circular convolution" (0-based): (x * y)_j = sum_i x_i y_{(j - i) mod n}
    n = len(x)
    return np.array([sum(x[i] * y[(j - i) % n] for i in range(n)) for j in range(n)])


def _circ_xcorr(x, y):
    # Def. "Circular cross-correlation" (0-based): (x * y)_j = sum_i conj(x_i) y_{(j + i) mod n}
    n = len(x)
    return np.array([sum(np.conj(x[i]) * y[(j + i) % n] for i in range(n)) for j in range(n)])


def test_convolution_theorem():
    rng = np.random.default_rng(5)
    m = 32
    x = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    y = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    assert np.allclose(oracle.fft(_circ_conv(x, y)), oracle.fft(x) * oracle.fft(y))
    assert np.allclose(oracle.fft(_circ_xcorr(x, y)), np.conj(oracle.fft(x)) * oracle.fft(y))


def test_first_component_of_inverse_is_mean():
    # e_1^T F^{-1}(x o conj(y)) = <x, y>/m, used in the proof of Lemma
    # "general-expectation-variance" (Eq. inner)
    rng = np.random.default_rng(6)
    m = 16
    x = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    y = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    inv = np.conj(oracle.fft(np.conj(x * np.conj(y)))) / m  # F^{-1} = conj(F conj(.)) / m
    assert np.isclose(inv[0], np.vdot(y, x) / m)
