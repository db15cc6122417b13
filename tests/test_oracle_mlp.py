"""Pins of the FP64 reference MLP (oracle/mlp.py) against facts that do not come
from the reference itself: finite differences, tabulated values of the normal
distribution, closed forms of Adam's first step and of least squares."""
import math

import numpy as np

from oracle import mlp


def test_gelu_against_tabulated_normal_cdf():
    # Phi(1) = 0.841344746068543, Phi(-1) = 0.158655253931457, Phi(2) = 0.977249868051821
    x = np.array([0.0, 1.0, -1.0, 2.0, 8.0])
    want = np.array([0.0, 0.841344746068543, -0.158655253931457, 2 * 0.977249868051821, 8.0])
    assert np.allclose(mlp.gelu(x), want, rtol=1e-13, atol=1e-13)
    # phi(1) = 0.241970724519143: gelu'(1) = Phi(1) + phi(1)
    assert math.isclose(float(mlp.gelu_grad(np.array([1.0]))[0]), 0.841344746068543 + 0.241970724519143,
                        rel_tol=1e-13)
    assert math.isclose(float(mlp.gelu_grad(np.array([0.0]))[0]), 0.5, rel_tol=1e-15)


def test_backprop_matches_central_differences():
    hidden = (5, 4, 3)
    n_in = 6
    rng = np.random.default_rng(3)
    theta = mlp.init_params(n_in, seed=7, hidden=hidden) + 0.1 * rng.standard_normal(mlp.n_params(n_in, hidden))
    Z = rng.standard_normal((9, n_in))
    y = rng.standard_normal(9)
    _, g = mlp.loss_and_grad(theta, Z, y, n_in, hidden)
    h = 1e-6
    num = np.empty_like(theta)
    for i in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        num[i] = (mlp.loss_and_grad(tp, Z, y, n_in, hidden)[0] - mlp.loss_and_grad(tm, Z, y, n_in, hidden)[0]) / (2 * h)
    assert np.allclose(g, num, rtol=1e-6, atol=1e-9)


def test_layout_and_sizes():
    assert mlp.n_params(9) == 9 * 128 + 128 + 2 * (128 * 128 + 128) + 128 + 1
    theta = np.arange(mlp.n_params(2, (3,)), dtype=float)
    (W1, b1), (W2, b2) = mlp.unpack(theta, 2, (3,))
    assert W1.shape == (3, 2) and list(W1.ravel()) == [0, 1, 2, 3, 4, 5] and list(b1) == [6, 7, 8]
    assert W2.shape == (1, 3) and list(W2.ravel()) == [9, 10, 11] and list(b2) == [12]


def test_adam_first_step_moves_each_weight_by_lr():
    # after one bias-corrected step m_hat = g and v_hat = g^2, so the move is lr * g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3])
    th, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), step=1, lr=0.01, eps=0.0)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=1e-12)


def test_output_layer_gradient_is_the_least_squares_gradient():
    # with the hidden weights fixed, the loss is quadratic in the output layer: its
    # gradient is (2/B) H^T (H w + b - y), the normal-equations residual
    n_in, hidden = 3, (4,)
    rng = np.random.default_rng(11)
    theta = mlp.init_params(n_in, seed=2, hidden=hidden)
    Z = rng.standard_normal((7, n_in))
    y = rng.standard_normal(7)
    (W1, b1), (W2, b2) = mlp.unpack(theta, n_in, hidden)
    H = mlp.gelu(Z @ W1.T + b1)
    r = H @ W2[0] + b2[0] - y
    _, g = mlp.loss_and_grad(theta, Z, y, n_in, hidden)
    gw2 = g[n_in * 4 + 4:n_in * 4 + 4 + 4]
    gb2 = g[-1]
    assert np.allclose(gw2, 2.0 / 7 * H.T @ r, rtol=1e-12)
    assert math.isclose(gb2, 2.0 / 7 * r.sum(), rel_tol=1e-12)
