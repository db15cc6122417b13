"""GPU parity of WLOG 1 (Sec. 4.1) inside the library: networks where a mode joins
two or more contractions (hyperedges) are given to tnsk_estimate as they are; the
library appends diagonal copy tensors and sketches their n nonzeros directly. The
oracle rewrites the same dtype-rounded tensors with dense copy tensors
(oracle.normalize.copy_tensors, the order the header states) and runs its method 1
(or its cross-correlation chain) with the same seeds: per-bin sketches, per-rep
estimates, plans and a turnstile stream are compared."""
import numpy as np
import pytest

import oracle
from oracle import prior
from oracle.normalize import copy_tensors
from paper_2603_07387_gb300 import tnsk
from paper_2603_07387_gb300 import workloads as W

from gpu_common import sketch_tol, TOL, assert_parity, gpu_estimate, gpu_network, rounded

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
    rng = np.random.default_rng(44)
    # the paper's example: b's single mode in two contractions, sum_i a(i) b(i) c(i)
    abc = W.NetSpec([rng.standard_normal(9) for _ in range(3)], [(0, 1), (1, 2)], [], "abc")
    # X(6,5) Y(5,6,4) Z(5,4,3): modes 0,1 | 2,3,4 | 5,6,7. Class {1, 2, 5} (mode 2 in two
    # contractions), class {0, 3} plain, class {4, 6} listed twice, open 7
    X, Y, Z = rng.standard_normal((6, 5)), rng.standard_normal((5, 6, 4)), rng.standard_normal((5, 4, 3))
    mixed = W.NetSpec([X, Y, Z], [(1, 2), (3, 0), (2, 5), (4, 6), (6, 4)], [7], "mixed")
    # a class of four modes with a redundant bracket, two open legs
    A, B, C = rng.standard_normal((7, 3)), rng.standard_normal((7, 7)), rng.standard_normal((2, 7))
    four = W.NetSpec([A, B, C], [(0, 2), (2, 3), (3, 5), (5, 0)], [4, 1], "four")
    return [abc, mixed, four]


def _oracle(spec, tdt, params, method):
    T, E, O = copy_tensors(rounded(spec, tdt), spec.edges, spec.open)
    if method == tnsk.CROSSCORR:
        y = prior.estimate(T, E, O, params.m, params.reps, params.seed)
        s = prior.estimate(T, E, O, params.m, params.reps, params.seed, abs_mode=True)
        return y, s
    return oracle.m1_estimate(T, E, O, m=params.m, reps=params.reps, seed=params.seed)


@pytest.mark.parametrize("prec", [tnsk.PREC_FP32, tnsk.PREC_FP64])
@pytest.mark.parametrize("m", [1, 16, 256])
def test_hyperedge_estimates(ctx, prec, m):
    tdt = torch.float64 if prec == tnsk.PREC_FP64 else torch.float32
    for spec in _specs():
        for method in (tnsk.GENERAL, tnsk.CROSSCORR):
            if method == tnsk.CROSSCORR and m > 16:
                continue  # the oracle's time-domain chain is O(m^2) per pair
            p = tnsk.Params(m=m, reps=5, seed=61, method=method, prec=prec)
            out, per = gpu_estimate(ctx, spec, p, tdt)
            y, s = _oracle(spec, tdt, p, method)
            assert_parity(per, y, s, TOL[prec], f"{spec.name} m={m} method={method}")


def test_hyperedge_sketches_per_bin(ctx):
    """tnsk_m1_sketch: the copy tensors' sketches follow the caller's tensors."""
    R, seed, m = 4, 17, 64
    for spec in _specs():
        X = rounded(spec, torch.float32)
        T, E, O = copy_tensors(X, spec.edges, spec.open)
        bins, signs = oracle.m1_tables(T, E, O, seed=seed, reps=R, m=m)
        want = oracle.m1_sketch(T, E, O, m, bins, signs)
        scale = oracle.m1_sketch(T, E, O, m, bins, signs, abs_mode=True)
        x = torch.zeros(want.shape, dtype=torch.float32, device="cuda")
        ctx.m1_sketch(gpu_network(spec, torch.float32), tnsk.Params(m=m, reps=R, seed=seed), x)
        ctx.sync()
        got = x.double().cpu().numpy()
        assert np.all(np.abs(got - want) <= sketch_tol(T, E, O, m, bins, signs, tnsk.PREC_FP32)), spec.name


def test_hyperedge_plans_and_streams(ctx):
    """A plan (graph replays) of the three networks, and a turnstile stream whose tensors
    start as all zeros and receive the entries as updates: the same estimates."""
    specs = _specs()
    params = [tnsk.Params(m=128, reps=6, seed=70 + i) for i in range(len(specs))]
    nets = [gpu_network(s, torch.float32) for s in specs]
    outs, pers = [], []
    for s in specs:
        dims = [d for x in s.tensors for d in np.shape(x)]
        o = int(np.prod([dims[g] for g in s.open])) if s.open else 1
        outs.append(torch.zeros(o, dtype=torch.float64, device="cuda"))
        pers.append(torch.zeros((6, o), dtype=torch.float64, device="cuda"))
    plan = ctx.plan(nets, params, outs, pers)
    for _ in range(3):
        plan.run()
        ctx.sync()
        for s, pr, pe in zip(specs, params, pers):
            y, sc = _oracle(s, torch.float32, pr, tnsk.GENERAL)
            assert_parity(pe.cpu().numpy(), y, sc, TOL[pr.prec], f"plan {s.name}")
    plan.close()
    s = specs[1]
    X = rounded(s, torch.float32)
    zeros = tnsk.Network([tnsk.Zeros(*np.shape(x)) for x in X], s.edges, s.open)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    per = torch.zeros((6, 3), dtype=torch.float64, device="cuda")
    st = ctx.stream(zeros, params[1], out, per)
    tk = np.concatenate([np.full(x.size, k, np.int32) for k, x in enumerate(X)])
    ti = np.concatenate([np.arange(x.size, dtype=np.int64) for x in X])
    dv = np.concatenate([x.reshape(-1) for x in X])
    st.update(torch.as_tensor(tk, device="cuda"), torch.as_tensor(ti, device="cuda"),
              torch.as_tensor(dv, dtype=torch.float64, device="cuda"))
    st.estimate()
    ctx.sync()
    y, sc = _oracle(s, torch.float32, params[1], tnsk.GENERAL)
    assert_parity(per.cpu().numpy(), y, sc, TOL[tnsk.PREC_FP32], "stream mixed")
    st.close()


def test_hyperedge_errors(ctx):
    """The acyclic method takes no hyperedges (TNSK_ERR_UNSUPPORTED); a class of 13
    modes exceeds the copy tensor's order limit."""
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    abc = _specs()[0]
    with pytest.raises(tnsk.TnskError) as e:
        ctx.estimate(gpu_network(abc, torch.float32), tnsk.Params(m=8, reps=2, method=tnsk.ACYCLIC), out)
    assert e.value.status == -3
    vs = [torch.ones(2, device="cuda") for _ in range(13)]
    with pytest.raises(tnsk.TnskError) as e:
        ctx.estimate(tnsk.Network(vs, [(0, k) for k in range(1, 13)], []), tnsk.Params(m=8, reps=2), out)
    assert e.value.status == -3
    ctx.sync()
