"""The row-sorted method-1 sketch of large FP32 tensors (at least 2^24 entries, a
contracted leading mode of 1024 .. 2^17 indices, m <= 2^14): rows visited in the
order of their leading-mode bins, one register sum per column and bin. Against the
oracle per bin (tnsk_m1_sketch) and per repetition (tnsk_estimate), including a
leading mode and rows that are not multiples of the CTA's sizes, an order-3 tensor,
and complemented leading modes, from m = 256 up to the form's largest m, 2^14."""
import numpy as np
import pytest

import oracle
from paper_2603_07387_gb300 import tnsk

from gpu_common import TOL, assert_parity, gpu_estimate, gpu_network, rounded, sketch_tol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tnsk.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def _specs():
    from paper_2603_07387_gb300 import workloads as W

    rng = np.random.default_rng(77)
    n = 4096
    A = rng.standard_normal((n, n)).astype(np.float32)
    B = rng.standard_normal((n, n)).astype(np.float32)
    # tr(AB): both leading modes are second endpoints of their contractions (complement)
    trab = W.NetSpec([A, B], [(1, 2), (3, 0)], [], "trAB")
    # an order-3 tensor of 3000 x 70 x 80 (16.8 M entries, rows of 5600: not a multiple
    # of the 512-column strips; leading mode a first endpoint) against three vectors
    X = rng.standard_normal((3000, 70, 80)).astype(np.float32)
    vs = [rng.standard_normal(d).astype(np.float32) for d in (3000, 70, 80)]
    order3 = W.NetSpec([X] + vs, [(0, 3), (4, 1), (2, 5)], [], "order3")
    return [trab, order3]


@pytest.mark.parametrize("m", [256, 4096, 16384])
def test_rowsort_sketch_per_bin(ctx, m):
    R, seed = 2, 0x7E57
    for spec in _specs():
        X = rounded(spec, torch.float32)
        bins, signs = oracle.m1_tables(X, spec.edges, spec.open, seed=seed, reps=R, m=m)
        want = oracle.m1_sketch(X, spec.edges, spec.open, m, bins, signs)
        x = torch.zeros(want.shape, dtype=torch.float32, device="cuda")
        ctx.m1_sketch(gpu_network(spec, torch.float32), tnsk.Params(m=m, reps=R, seed=seed), x)
        ctx.sync()
        got = x.double().cpu().numpy()
        bound = sketch_tol(X, spec.edges, spec.open, m, bins, signs, tnsk.PREC_FP32)
        assert np.all(np.abs(got - want) <= bound), spec.name


def test_rowsort_estimates(ctx):
    for spec in _specs():
        p = tnsk.Params(m=1024, reps=2, seed=5)
        _, per = gpu_estimate(ctx, spec, p, torch.float32)
        X = rounded(spec, torch.float32)
        y, s = oracle.m1_estimate(X, spec.edges, spec.open, m=p.m, reps=p.reps, seed=p.seed)
        assert_parity(per, y, s, TOL[tnsk.PREC_FP32], spec.name)
