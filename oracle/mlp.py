"""FP64 reference of the learned sketch-size predictor (test infrastructure only).

A multilayer perceptron F -> 128 -> 128 -> 128 -> 1 with GELU (the exact, erf form
x Phi(x)) after each hidden layer, trained on a mean squared error by Adam. The GPU
path (libtnsk's tnsk_mlp_* calls) is compared with these functions on the same
parameters and batches; only tests/ may import this module.

Parameter layout (shared with the GPU as a contract, not as code): for each layer l,
W_l [n_out][n_in] row-major then b_l [n_out], layers in order, all in one flat
vector. Inputs are standardised first: z = (x - mu) / sigma per feature.
"""
from __future__ import annotations

import math

import numpy as np

HIDDEN = (128, 128, 128)


def layer_shapes(n_in: int, hidden=HIDDEN):
    dims = [n_in, *hidden, 1]
    return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]


def n_params(n_in: int, hidden=HIDDEN) -> int:
    return sum(o * i + o for o, i in layer_shapes(n_in, hidden))


def unpack(theta, n_in: int, hidden=HIDDEN):
    """Flat parameter vector -> [(W, b), ...]."""
    out, off = [], 0
    for o, i in layer_shapes(n_in, hidden):
        W = theta[off:off + o * i].reshape(o, i)
        off += o * i
        b = theta[off:off + o]
        off += o
        out.append((W, b))
    return out


_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    """d/dx [x Phi(x)] = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(theta, Z, n_in: int, hidden=HIDDEN):
    """Z: [B][n_in] standardised inputs. Returns (y [B], cache of (input, pre-activation))."""
    h = np.asarray(Z, dtype=np.float64)
    cache = []
    layers = unpack(np.asarray(theta, dtype=np.float64), n_in, hidden)
    for li, (W, b) in enumerate(layers):
        pre = h @ W.T + b
        cache.append((h, pre))
        h = gelu(pre) if li < len(layers) - 1 else pre
    return h[:, 0], cache


def loss_and_grad(theta, Z, y, n_in: int, hidden=HIDDEN):
    """Mean squared error L = (1/B) sum (f(z_b) - y_b)^2 and dL/dtheta (backpropagation)."""
    out, cache = forward(theta, Z, n_in, hidden)
    B = len(y)
    diff = out - np.asarray(y, dtype=np.float64)
    loss = float(np.mean(diff * diff))
    layers = unpack(np.asarray(theta, dtype=np.float64), n_in, hidden)
    grads = []
    d = (2.0 / B) * diff[:, None]  # dL/d(pre-activation) of the output layer
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        h_in, _ = cache[li]
        gW = d.T @ h_in
        gb = d.sum(axis=0)
        grads.append((gW, gb))
        if li > 0:
            _, pre_prev = cache[li - 1]
            d = (d @ W) * gelu_grad(pre_prev)
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def adam_step(theta, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), bias-corrected; returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def init_params(n_in: int, seed: int, hidden=HIDDEN):
    """He-style uniform initialisation: W ~ U(-a, a), a = sqrt(6 / n_in_layer), b = 0."""
    rng = np.random.default_rng(seed)
    parts = []
    for o, i in layer_shapes(n_in, hidden):
        a = math.sqrt(6.0 / i)
        parts.append(rng.uniform(-a, a, size=o * i))
        parts.append(np.zeros(o))
    return np.concatenate(parts)
