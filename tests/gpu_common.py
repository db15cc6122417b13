"""Helpers shared by the GPU parity tests: run a spec through libtnsk (C ABI) and
through the oracle on the same (dtype-rounded) inputs and seeded tables."""
import numpy as np

import oracle
from paper_2603_07387_gb300 import tnsk
from paper_2603_07387_gb300 import workloads as W

TOL = {tnsk.PREC_FP32: 1e-5, tnsk.PREC_FP64: 1e-10}


def rounded(spec, torch_dtype):
    """The spec's tensors rounded to torch_dtype (what the GPU reads), as float64 numpy."""
    ts = W.to_torch(spec, device="cpu", dtype=torch_dtype)
    return [t.double().numpy() for t in ts]


def gpu_network(spec, torch_dtype):
    return tnsk.Network(W.to_torch(spec, device="cuda", dtype=torch_dtype), spec.edges, spec.open)


def gpu_estimate(ctx, spec, params, torch_dtype):
    import torch

    net = gpu_network(spec, torch_dtype)
    dims = [d for x in spec.tensors for d in np.shape(x)]
    O = int(np.prod([dims[g] for g in spec.open])) if spec.open else 1
    out = torch.zeros(max(O, 1), dtype=torch.float64, device="cuda")
    per = torch.zeros((params.reps, max(O, 1)), dtype=torch.float64, device="cuda")
    ctx.estimate(net, params, out, per)
    ctx.sync()
    return out.cpu().numpy()[:O], per.cpu().numpy()[:, :O]


def oracle_estimate(spec, params, torch_dtype):
    X = rounded(spec, torch_dtype)
    if params.method == tnsk.GENERAL:
        y, s = oracle.m1_estimate(X, spec.edges, spec.open, m=params.m, reps=params.reps, seed=params.seed)
    else:
        root = params.root
        if root < 0:
            sizes = [x.size for x in X]
            root = int(np.argmin(sizes))
        y, s = oracle.m2_estimate(X, spec.edges, m=params.m, reps=params.reps, seed=params.seed, root=root)
        y, s = y[:, None], s[:, None]
    return y, s


def assert_parity(gpu_per_rep, orc_y, orc_s, tol, what=""):
    """|y_gpu - y_oracle| <= tol * S per rep and entry, S the oracle's cancellation-aware
    scale (sum of the magnitudes the estimate is built from)."""
    err = np.abs(gpu_per_rep - orc_y)
    bound = tol * np.maximum(orc_s, 1e-300)
    bad = err > bound
    if bad.any():
        i = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: parity off at {tuple(i)}: gpu {gpu_per_rep[tuple(i)]!r} "
                             f"oracle {orc_y[tuple(i)]!r} scale {orc_s[tuple(i)]!r} "
                             f"({bad.sum()} of {bad.size} entries beyond {tol})")
