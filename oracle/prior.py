"""The earlier cross-correlation estimator that Sec. 4.2 contrasts with method 1, in
FP64 numpy (test infrastructure only: the tests, the smoke check and the
benchmark's CPU-baseline leg are the only callers).

Every contraction e gets one count sketch C_e (the same table as method 1's edge e:
hash contract, table id (1 << 56) | e), every tensor its plain tensor sketch
x_k = (C_{e_1} (x) ... ) vec(X_k) (bin sum of h_e over its contracted modes mod m,
sign product; one m-vector per open index), and the sketches are combined by the
circular cross-correlation x_1 * x_2 * ... * x_p taken left to right, of which the
first component (e_1) is the estimate (the two examples of the prior method in
Sec. 4.2). Cross-correlation is written out in the time domain:
(a * b)(k) = sum_j a(j) b((j + k) mod m). No complement count sketch is used, so a
contraction whose two tensors are both, or neither, conjugated by the chain (an odd
cycle always has one) is not estimated without bias: on the triangle tr(XYZ) the
expectation is tc * P(2 h(i) = 0 mod m), about 2 tc / m.
"""
from __future__ import annotations

import numpy as np

from . import count_sketch, tid


def _sketch(x, k, off, edges, tabs, m, abs_mode=False):
    """Plain tensor sketch of tensor k: [O_k, m] (open index row-major in mode order);
    abs_mode: |X| with every sign +1 (the magnitudes the estimate is built from)."""
    x = np.asarray(x, dtype=np.float64)
    if abs_mode:
        x = np.abs(x)
    q = x.ndim
    edge_of = {}
    for e, (u, v) in enumerate(edges):
        edge_of[u] = e
        edge_of[v] = e
    modes = range(off[k], off[k] + q)
    open_dims = [x.shape[g - off[k]] for g in modes if g not in edge_of]
    O = int(np.prod(open_dims)) if open_dims else 1
    out = np.zeros((O, m))
    for idx in np.ndindex(*x.shape) if q else [()]:
        b, s, o = 0, 1, 0
        for d, g in enumerate(modes):
            if g in edge_of:
                bins, signs = tabs[edge_of[g]]
                b += int(bins[idx[d]])
                s *= 1 if abs_mode else int(signs[idx[d]])
            else:
                o = o * x.shape[d] + idx[d]
        out[o, b % m] += s * float(x[idx])
    return out


def _xcorr(a, b):
    m = a.shape[0]
    return np.array([sum(a[j] * b[(j + k) % m] for j in range(m)) for k in range(m)])


def estimate(tensors, edges, open_modes, m: int, reps: int, seed: int, abs_mode: bool = False):
    """Per-rep estimates y[R, O] of the cross-correlation estimator (O = product of
    the open dims in open_modes order; 1 for a full network). abs_mode: the same
    chain on magnitude sketches, a bound on the sum of the magnitudes of the terms
    (the scale of a rounding-error tolerance)."""
    off = [0]
    for x in tensors:
        off.append(off[-1] + np.ndim(x))
    dims = [d for x in tensors for d in np.shape(x)]
    O = int(np.prod([dims[g] for g in open_modes])) if open_modes else 1
    y = np.zeros((reps, O))
    for r in range(reps):
        tabs = [count_sketch(seed, r, tid(1, e), dims[u], m) for e, (u, v) in enumerate(edges)]
        sk = [_sketch(x, k, off, edges, tabs, m, abs_mode) for k, x in enumerate(tensors)]
        for o, oidx in enumerate(np.ndindex(*[dims[g] for g in open_modes]) if open_modes else [()]):
            # each tensor's open index from the output multi-index, row-major in its mode order
            at = dict(zip(open_modes, oidx))
            acc = None
            for k in range(len(tensors)):
                ok = 0
                for g in range(off[k], off[k + 1]):
                    if g in at:
                        ok = ok * dims[g] + at[g]
                v = sk[k][ok]
                acc = v if acc is None else _xcorr(acc, v)
            y[r, o] = acc[0]
    return y
