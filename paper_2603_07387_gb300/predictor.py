"""The learned sketch-size predictor: measuring training samples, training, choosing m.

A sample is (features of a network at sketch size m and R reps, log10 of the
relative error |y - tc| / |tc| of one method-1 estimate). The estimates run in
libtnsk (one batch per (m, R, seed)); the exact values tc are the caller's input
(the tests take them from the FP64 oracle), so nothing here computes a
contraction itself. Training and inference run in libtnsk's kernels
(tnsk_mlp_train / tnsk_mlp_predict); tnsk_choose_params picks m.

Networks for training follow the grid family of the benchmark: L1 x L2 sites with
L1 in 1..4, L2 in 2..4, bond 2..8, entries U(0, 1), m in 2^6 .. 2^16.
"""
from __future__ import annotations

import numpy as np

from . import tnsk
from . import workloads as W

LOG2M = tuple(range(6, 17))


def grid_specs(rng, count: int):
    """`count` random grids of the training family (seeded by rng)."""
    specs = []
    for _ in range(count):
        L1 = int(rng.integers(1, 5))
        L2 = int(rng.integers(2, 5))
        bond = int(rng.integers(2, 9))
        specs.append(W.grid(L1, L2, bond, seed=int(rng.integers(1 << 31))))
    return specs


def measure(ctx, specs, exact, log2ms=LOG2M, reps=(4, 16), seeds=(1, 2), device="cuda",
            max_bytes: float = 4e9):
    """Samples (X [n][9] float32, y [n] float32) for every spec x m x R x seed: one
    libtnsk estimate per sample against exact[i] = tc of specs[i]. Networks run in
    batches whose sketches and spectra stay below about max_bytes."""
    import torch

    nets = [tnsk.Network(W.to_torch(s, device, torch.float32), s.edges, s.open) for s in specs]
    base = [ctx.features(n, tnsk.Params(m=1, reps=1)) for n in nets]
    exact = np.asarray(exact, dtype=np.float64)
    pmax = max(len(s.tensors) for s in specs)
    X, y = [], []
    for l in log2ms:
        for R in reps:
            # sketch + spectra per network: about 12 bytes per bin, rep and tensor
            chunk = int(max(1, max_bytes // (12.0 * R * pmax * (1 << l))))
            for sd in seeds:
                params = [tnsk.Params(m=1 << l, reps=R, seed=int(sd) * 1000003 + i) for i in range(len(nets))]
                outd = torch.zeros(len(nets), dtype=torch.float64, device=device)
                outs = [outd[i:i + 1] for i in range(len(nets))]
                for c0 in range(0, len(nets), chunk):
                    ctx.estimate_batch(nets[c0:c0 + chunk], params[c0:c0 + chunk], outs[c0:c0 + chunk])
                ctx.sync()
                est = outd.cpu().numpy()
                rel = np.abs(est - exact) / np.abs(exact)
                for i, b in enumerate(base):
                    f = b.copy()
                    f[7] = l
                    f[8] = np.log2(R)
                    X.append(f)
                    y.append(np.log10(max(rel[i], 1e-12)))
    return np.asarray(X, dtype=np.float32), np.asarray(y, dtype=np.float32)


def train(ctx, X, y, epochs: int = 200, batch: int = 256, lr: float = 1e-3, seed: int = 0, device="cuda"):
    """A fresh predictor trained on the samples; returns (Mlp, final mean squared error)."""
    import torch

    mlp = tnsk.Mlp(ctx, seed=seed)
    Xd = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float32), device=device)
    yd = torch.as_tensor(np.ascontiguousarray(y, dtype=np.float32), device=device)
    loss = mlp.train(Xd, yd, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return mlp, loss


def choose(ctx, net, target_err: float, reps: int, mlp=None, seed: int = 0):
    """(params with the chosen m, predicted error), or (None, best predicted error)
    when no m <= 2^16 meets the target."""
    return ctx.choose_params(net, target_err, tnsk.Params(m=1, reps=reps, seed=seed), mlp)
