"""GPU parity of the earlier cross-correlation estimator (TNSK_CROSSCORR, Sec. 4.2's
prior method) against the oracle's time-domain cross-correlation chain: per-rep
estimates on an acyclic chain, the cyclic triangle of the paper's example, a ring of
four tensors and a pair with open legs, FP32 and FP64, same seeds. Tolerance as the
other parity tests, scaled by the chain on magnitude sketches."""
import numpy as np
import pytest

from oracle import prior
from paper_2603_07387_gb300 import tnsk
from paper_2603_07387_gb300 import workloads as W

from gpu_common import TOL, assert_parity, gpu_estimate, rounded

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
    rng = np.random.default_rng(12)
    chain = W.NetSpec([rng.standard_normal(7), rng.standard_normal((7, 5)), rng.standard_normal(5)],
                      [(0, 1), (2, 3)], [], "chain")
    tri = W.NetSpec([rng.standard_normal((4, 6)), rng.standard_normal((6, 5)), rng.standard_normal((5, 4))],
                    [(1, 2), (3, 4), (5, 0)], [], "triangle")
    A, B, C, D = rng.standard_normal((3, 4)), rng.standard_normal((4, 3)), rng.standard_normal((3, 4)), \
        rng.standard_normal((4, 3))
    ring = W.NetSpec([A, B, C, D], [(1, 2), (3, 4), (5, 6), (7, 0)], [], "ring4")
    open_pair = W.NetSpec([rng.standard_normal((3, 6)), rng.standard_normal((6, 2))], [(1, 2)], [3, 0], "open")
    return [chain, tri, ring, open_pair]


@pytest.mark.parametrize("prec", [tnsk.PREC_FP32, tnsk.PREC_FP64])
@pytest.mark.parametrize("m", [1, 16, 64])
def test_crosscorr_matches_the_oracle(ctx, prec, m):
    tdt = torch.float64 if prec == tnsk.PREC_FP64 else torch.float32
    for spec in _specs():
        p = tnsk.Params(m=m, reps=4, seed=21, method=tnsk.CROSSCORR, prec=prec)
        out, per = gpu_estimate(ctx, spec, p, tdt)
        X = rounded(spec, tdt)
        y = prior.estimate(X, spec.edges, spec.open, m, p.reps, p.seed)
        s = prior.estimate(X, spec.edges, spec.open, m, p.reps, p.seed, abs_mode=True)
        assert_parity(per, y, s, TOL[prec], f"{spec.name} m={m}")


def test_crosscorr_refused_where_it_has_no_meaning(ctx):
    spec = _specs()[0]
    net = tnsk.Network(W.to_torch(spec, device="cuda", dtype=torch.float32), spec.edges, spec.open)
    p = tnsk.Params(m=64, reps=4, method=tnsk.CROSSCORR)
    with pytest.raises(tnsk.TnskError) as e:
        ctx.choose_params(net, 0.1, p)
    assert e.value.status == -3
