"""Small seeded runs of the hot path, one workload each, for profiler captures and
quick timing of single kernels. Each case plans one batch, runs it three times to warm
up, then three times with libtnsk's per-kernel CUDA-event profile on and prints the
mean time per run of the kernel the case is about and its algorithmic bytes per
second.

    python -m paper_2603_07387_gb300.cases chains  [--count 16] [--prec fp32|bf16]
        method 2 (Algorithm 4) on `count` merged tensor-train chains (vector, six
        1024 x 1024 matrices, vector), m = 1024, 64 reps: the sketched product
        (m2_gemm_tc_stream_kernel, or m2_gemm_bf16_kernel for BF16 storage).
    python -m paper_2603_07387_gb300.cases rungs   [--count 64]
        method 2 on `count` tensor-train pair chains (8 sites, bond 32, physical 8)
        with the six inner sites as grouped tensors (tnsk.Rung), m = 1024, 64 reps:
        the factored product on the tensor cores (m2_rung_tc_kernel after
        m2_rung_prep_kernel); rate in TFLOP/s of one pass of the two contractions.
    python -m paper_2603_07387_gb300.cases trace4  [--n 4096] [--reps 1]
        method 1 (Algorithm 3) on tr(ABCD) of four n x n FP32 N(0,1) matrices,
        m = 4096: the row-sorted sketch (m1_rowsort_kernel) when reps <= 2, the
        fixed-point scatter otherwise.
    python -m paper_2603_07387_gb300.cases ladders [--count 8]
        method 1 on `count` tensor-train ladders (two chains of 8 cores, bond 32,
        physical 8), m = 1024, 64 reps: the fixed-point scatter (m1_scatter_fx_kernel).
    python -m paper_2603_07387_gb300.cases grid [--log2m 14] [--reps 256]
        method 1 on the cyclic 4 x 4 grid of bond 8 (U(0,1), FP32): the transforms and
        the product of the spectra (m1_fft_mid_kernel at 2^11 <= m <= 2^14,
        m1_fft_large_kernel above).
"""
from __future__ import annotations

import argparse

from . import tnsk
from . import workloads as W


def _run(ctx, nets, params, outs, key, nbytes, flops=None):
    plan = ctx.plan(nets, params, outs)
    for _ in range(3):
        plan.run()
    ctx.sync()
    ctx.profile(True)
    for _ in range(3):
        plan.run()
    prof = ctx.profile_read()
    ctx.profile(False)
    plan.close()
    ms, launches = prof[key]
    per_run = ms / 3
    if flops is not None:
        print(f"{key}: {per_run:.4f} ms per run ({launches // 3} launches), "
              f"{flops / (per_run / 1e3) / 1e12:.2f} TFLOP/s")
    else:
        print(f"{key}: {per_run:.4f} ms per run ({launches // 3} launches), "
              f"{nbytes / (per_run / 1e3) / 1e9:.1f} GB/s of algorithmic bytes")


def chains(ctx, count: int, prec: str):
    import torch

    dt = torch.bfloat16 if prec == "bf16" else torch.float32
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    edges = [(0, 1)] + [(2 * k, 2 * k + 1) for k in range(1, 7)]
    nets, outs = [], []
    for _ in range(count):
        ts = [torch.randn(1024, generator=g, device="cuda").to(dt)]
        ts += [(torch.randn(1024, 1024, generator=g, device="cuda") / 32).to(dt) for _ in range(6)]
        ts += [torch.randn(1024, generator=g, device="cuda").to(dt)]
        nets.append(tnsk.Network(ts, edges, []))
        outs.append(torch.zeros(1, dtype=torch.float64, device="cuda"))
    p = tnsk.PREC_BF16 if prec == "bf16" else tnsk.PREC_FP32
    params = [tnsk.Params(m=1024, reps=64, seed=7, method=tnsk.ACYCLIC, prec=p) for _ in nets]
    # X of every interior matrix is read once per launch (one height per launch)
    _run(ctx, nets, params, outs, "m2_gemm", 6 * count * 1024 * 1024 * dt.itemsize)


def rungs(ctx, count: int):
    import torch

    nets, outs = [], []
    for i in range(count):
        A, B = W.tt_cores(seed=20260307 + i)
        spec = W.tt_chain(A, B)
        ts = [torch.as_tensor(spec.tensors[0], dtype=torch.float32, device="cuda")]
        ts += [tnsk.Rung(torch.as_tensor(A[k], dtype=torch.float32, device="cuda"),
                         torch.as_tensor(B[k], dtype=torch.float32, device="cuda")) for k in range(1, 7)]
        ts.append(torch.as_tensor(spec.tensors[-1], dtype=torch.float32, device="cuda"))
        nets.append(tnsk.Network(ts, spec.edges, []))
        outs.append(torch.zeros(1, dtype=torch.float64, device="cuda"))
    params = [tnsk.Params(m=1024, reps=64, seed=7, method=tnsk.ACYCLIC, root=0) for _ in nets]
    # per grouped site and rep: two contractions of 2 s n^3 = 2 x 8 x 32^3 FLOPs each
    _run(ctx, nets, params, outs, "m2_gemm", 0, flops=6 * count * 64 * 2 * 2 * 8 * 32 ** 3)


def trace4(ctx, n: int, reps: int):
    import torch

    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    mats = [torch.randn((n, n), generator=g, device="cuda", dtype=torch.float32) for _ in range(4)]
    net = tnsk.Network(mats, [(1, 2), (3, 4), (5, 6), (7, 0)], [])
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    _run(ctx, [net], [tnsk.Params(m=4096, reps=reps, seed=0x7E57)], [out], "m1_scatter", 4 * n * n * 4)


def ladders(ctx, count: int):
    import torch

    nets, outs, params, nbytes = [], [], [], 0
    for i in range(count):
        A, B = W.tt_cores(seed=20260307 + i)
        spec = W.tt_ladder(A, B)
        ts = W.to_torch(spec, "cuda", torch.float32)
        nbytes += sum(t.numel() * 4 for t in ts)
        nets.append(tnsk.Network(ts, spec.edges, spec.open))
        outs.append(torch.zeros(1, dtype=torch.float64, device="cuda"))
        params.append(tnsk.Params(m=1024, reps=64, seed=0x7E57))
    _run(ctx, nets, params, outs, "m1_scatter", nbytes)


def grid(ctx, log2m: int, reps: int):
    import torch

    spec = W.grid(4, 4, 8)
    ts = W.to_torch(spec, "cuda", torch.float32)
    net = tnsk.Network(ts, spec.edges, spec.open)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # the transforms read every sketch once (4 bytes per bin, 16 sketches per rep)
    _run(ctx, [net], [tnsk.Params(m=1 << log2m, reps=reps, seed=W.HASH_SEED)], [out], "m1_spectrum",
         16 * reps * (1 << log2m) * 4)


def main(argv=None):
    import torch

    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("case", choices=("chains", "rungs", "trace4", "ladders", "grid"))
    ap.add_argument("--log2m", type=int, default=14)
    ap.add_argument("--count", type=int, default=None)
    ap.add_argument("--prec", choices=("fp32", "bf16"), default="fp32")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--reps", type=int, default=None)
    a = ap.parse_args(argv)
    ctx = tnsk.Context(0, torch.cuda.current_stream().cuda_stream)
    if a.case == "chains":
        chains(ctx, a.count or 16, a.prec)
    elif a.case == "rungs":
        rungs(ctx, a.count or 64)
    elif a.case == "trace4":
        trace4(ctx, a.n, a.reps or 1)
    elif a.case == "grid":
        grid(ctx, a.log2m, a.reps or 256)
    else:
        ladders(ctx, a.count or 8)
    ctx.close()


if __name__ == "__main__":
    main()
