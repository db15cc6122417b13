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


def sketch_tol(X, edges, open_modes, m, bins, signs, prec):
    """Per-bin bound on |GPU sketch - oracle sketch| for tnsk_m1_sketch's layout.
    FP64: 1e-12 of the sum of the bin's |entries|. FP32: 1e-6 of that sum (rounding of
    FP32 sums) plus the fixed-point quantisation of the privatised bins: every entry
    is rounded to a multiple of 2^-S with sum|x| 2^S <= 2^30 over its batch, an error
    of at most 2^-30 sum|x| of the batch, bounded here by 2^-30 ||X_k||_1 of its
    tensor, times the number of entries the bin receives."""
    scale = oracle.m1_sketch(X, edges, open_modes, m, bins, signs, abs_mode=True)
    if prec == tnsk.PREC_FP64:
        return 1e-12 * np.maximum(scale, 1e-300)
    ones = [np.ones_like(np.asarray(x, dtype=np.float64)) for x in X]
    counts = oracle.m1_sketch(ones, edges, open_modes, m, bins, signs, abs_mode=True)
    quant = np.zeros_like(scale)
    off = 0
    dims = [d for x in X for d in np.shape(x)]
    mode0 = 0
    for x in X:
        q = np.ndim(x)
        O = int(np.prod([dims[g] for g in open_modes if mode0 <= g < mode0 + q])) if q else 1
        quant[:, off:off + O * m] = 2.0**-30 * np.abs(np.asarray(x, dtype=np.float64)).sum()
        off += O * m
        mode0 += q
    return 1e-6 * np.maximum(scale, 1e-300) + counts * quant


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
