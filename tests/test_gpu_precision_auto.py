"""TNSK_PREC_AUTO against the oracle: the FP32 path, and the FP64 path for the reps whose
FP32 transforms may be inexact.

Every closed-network spectral kernel also returns the rep's magnitude sum
A_r = (1/m) sum_j |prod_k F x_k(j)|. FP32 rounding of the transforms and products is at
most about (p + 2 log2 m + 8) 2^-24 A_r, so a rep whose value y_r is far below A_r (its
sketches' spectra cancel in the sum: a high dynamic range) is recomputed in FP64 from
the same inputs with the same hash functions. Checked here:
- on a 2 x 2 grid of U(0,1) tensors (no cancellation) AUTO takes no rep in FP64 and returns
  the FP32 path's per-rep values exactly;
- on a pair of vectors whose two large entries cancel in the inner product (u = (L, L,
  ...), v = (L, -L, ...), L = 4096), at sizes of every spectral path (m = 32: block
  kernel; 256: warp kernel; 4096: per-sketch mid path; 2^15: two-pass large path),
  the FP32 path misses the oracle's per-rep values by more than 2^-17 of the values
  themselves on some rep, AUTO takes reps in FP64 and every AUTO per-rep value is
  within 2^-17 of the oracle's, relative to the value (plus the FP64 tolerance of the
  oracle's cancellation-aware scale);
- AUTO outside its scope (batches, open legs, method 2) is refused.
"""
import numpy as np
import pytest

from paper_2603_07387_gb300 import tnsk
from paper_2603_07387_gb300 import workloads as W

from gpu_common import TOL, gpu_estimate, gpu_network, oracle_estimate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 2.0 ** -17  # AUTO's per-rep target, relative to the value


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tnsk.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def _cancelling_pair(L=4096.0, n=64, seed=5):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    v = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    u[0], v[0], u[1], v[1] = L, L, L, -L
    return W.NetSpec([u, v], [(0, 1)], [], "cancelling-pair")


def test_auto_is_fp32_without_cancellation(ctx):
    spec = W.grid(2, 2, 4, seed=2)
    p32 = tnsk.Params(m=1024, reps=8, seed=9)
    pa = tnsk.Params(m=1024, reps=8, seed=9, prec=tnsk.PREC_AUTO)
    out32, per32 = gpu_estimate(ctx, spec, p32, torch.float32)
    outa, pera = gpu_estimate(ctx, spec, pa, torch.float32)
    n64, bound = ctx.auto_report()
    assert n64 == 0
    assert bound <= REL
    np.testing.assert_array_equal(pera, per32)
    np.testing.assert_array_equal(outa, out32)


@pytest.mark.parametrize("m", [32, 256, 4096, 1 << 15])
def test_auto_takes_fp64_where_fp32_cancels(ctx, m):
    spec = _cancelling_pair()
    R = 16
    y, s = oracle_estimate(spec, tnsk.Params(m=m, reps=R, seed=3), torch.float32)
    y, s = y[:, 0], s[:, 0]
    allowed = REL * np.abs(y) + TOL[tnsk.PREC_FP64] * s
    _, per32 = gpu_estimate(ctx, spec, tnsk.Params(m=m, reps=R, seed=3), torch.float32)
    assert (np.abs(per32[:, 0] - y) > allowed).any(), "the FP32 path should need FP64 here"
    outa, pera = gpu_estimate(ctx, spec, tnsk.Params(m=m, reps=R, seed=3, prec=tnsk.PREC_AUTO), torch.float32)
    n64, bound = ctx.auto_report()
    assert n64 > 0
    assert bound <= REL
    err = np.abs(pera[:, 0] - y)
    assert (err <= allowed).all(), f"m={m}: AUTO off at reps {np.nonzero(err > allowed)[0]}"
    # the estimate is the mean of the per-rep values (groups = 1)
    assert abs(outa[0] - pera[:, 0].mean()) <= 1e-12 * np.abs(pera[:, 0]).sum()


def test_auto_scope(ctx):
    spec = _cancelling_pair()
    net = gpu_network(spec, torch.float32)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    pa = tnsk.Params(m=256, reps=4, seed=1, prec=tnsk.PREC_AUTO)
    with pytest.raises(tnsk.TnskError) as e:  # batches
        ctx.estimate_batch([net, net], [pa, pa], [out, out])
    assert e.value.status == -3
    with pytest.raises(tnsk.TnskError) as e:  # method 2
        ctx.estimate(net, tnsk.Params(m=256, reps=4, seed=1, prec=tnsk.PREC_AUTO, method=tnsk.ACYCLIC), out)
    assert e.value.status == -3
    opened = W.NetSpec([spec.tensors[0], np.ones((64, 3))], [(0, 1)], [2], "open")
    with pytest.raises(tnsk.TnskError) as e:  # open legs
        ctx.estimate(gpu_network(opened, torch.float32), pa, torch.zeros(3, dtype=torch.float64, device="cuda"))
    assert e.value.status == -3
