"""Method 2 with open legs (Corollary "full-to-partial-tc"): every output entry, row-
major over the open list, is the full method-2 estimate of the network whose tensors
are sliced at that entry's open indices. Checked per rep and entry against the
oracle's method 2 on the sliced networks (numpy slicing, modes renumbered, the same
seed, the default root taken on the slices), in FP32 and FP64, for a chain with open
ends listed in reverse order, a star with open modes on a leaf and on the centre, and
a tensor with two open modes listed out of order; the combined output is the mean of
the per-rep values; plans refuse open legs for method 2."""
import numpy as np
import pytest

import oracle
from paper_2603_07387_gb300 import tnsk
from paper_2603_07387_gb300 import workloads as W

from gpu_common import TOL, assert_parity, gpu_estimate, gpu_network, rounded

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
    rng = np.random.default_rng(8)
    g = lambda *s: rng.standard_normal(s).astype(np.float32)  # noqa: E731
    chain = W.NetSpec([g(6, 5), g(5, 7), g(7, 4)], [(1, 2), (3, 4)], [5, 0], "chain, open ends reversed")
    # centre D (3, 5, 6, 2) with its last mode open; E (3, 4) with its second mode open
    star = W.NetSpec([g(3, 5, 6, 2), g(3, 4), g(5), g(6)], [(0, 4), (1, 6), (2, 7)], [3, 5], "star")
    two = W.NetSpec([g(2, 3, 5), g(5, 4)], [(2, 3)], [4, 1, 0], "two open modes on one tensor")
    return [chain, star, two]


def _sliced(X, edges, open_modes, o):
    """The tensors at output entry o (row-major over open_modes) and the renumbered edges."""
    dims = [d for x in X for d in np.shape(x)]
    offs = np.cumsum([0] + [np.ndim(x) for x in X])
    idx, rem = {}, o
    for gm in reversed(open_modes):
        idx[gm] = rem % dims[gm]
        rem //= dims[gm]
    out = []
    for k, x in enumerate(X):
        sl = tuple(idx[gm] if gm in idx else slice(None) for gm in range(offs[k], offs[k + 1]))
        out.append(np.ascontiguousarray(np.asarray(x)[sl]))
    new_id, c = {}, 0
    for gm in range(offs[-1]):
        if gm not in idx:
            new_id[gm] = c
            c += 1
    return out, [(new_id[u], new_id[v]) for u, v in edges]


@pytest.mark.parametrize("prec,tdt", [(tnsk.PREC_FP32, "float32"), (tnsk.PREC_FP64, "float64")])
def test_method2_open_legs_per_entry(ctx, prec, tdt):
    dt = getattr(torch, tdt)
    for spec in _specs():
        p = tnsk.Params(m=256, reps=8, seed=0x5EED, method=tnsk.ACYCLIC, prec=prec)
        out, per = gpu_estimate(ctx, spec, p, dt)
        X = rounded(spec, dt)
        dims = [d for x in X for d in np.shape(x)]
        O = int(np.prod([dims[gm] for gm in spec.open]))
        assert per.shape == (8, O)
        for o in range(O):
            Xs, es = _sliced(X, spec.edges, list(spec.open), o)
            root = int(np.argmin([x.size for x in Xs]))
            y, s = oracle.m2_estimate(Xs, es, m=p.m, reps=p.reps, seed=p.seed, root=root)
            assert_parity(per[:, o], y, s, TOL[prec], f"{spec.name} entry {o}")
        np.testing.assert_allclose(out, per.mean(axis=0), rtol=1e-12, atol=0)


def test_method2_open_legs_in_a_batch_and_not_in_plans(ctx):
    chain, star, _ = _specs()
    p = tnsk.Params(m=128, reps=4, seed=11, method=tnsk.ACYCLIC)
    p1 = tnsk.Params(m=128, reps=4, seed=11, method=tnsk.GENERAL)
    nets = [gpu_network(chain, torch.float32), gpu_network(star, torch.float32), gpu_network(chain, torch.float32)]
    outs = [torch.zeros(24, dtype=torch.float64, device="cuda"), torch.zeros(8, dtype=torch.float64, device="cuda"),
            torch.zeros(24, dtype=torch.float64, device="cuda")]
    pers = [torch.zeros((4, 24), dtype=torch.float64, device="cuda"),
            torch.zeros((4, 8), dtype=torch.float64, device="cuda"),
            torch.zeros((4, 24), dtype=torch.float64, device="cuda")]
    # method 2 on the chain and the star, method 1 on the chain, one batch
    ctx.estimate_batch(nets, [p, p, p1], outs, pers)
    ctx.sync()
    for spec, pp, per in ((chain, p, pers[0]), (star, p, pers[1])):
        got = per.cpu().numpy()
        X = rounded(spec, torch.float32)
        for o in range(got.shape[1]):
            Xs, es = _sliced(X, spec.edges, list(spec.open), o)
            y, s = oracle.m2_estimate(Xs, es, m=pp.m, reps=pp.reps, seed=pp.seed,
                                      root=int(np.argmin([x.size for x in Xs])))
            assert_parity(got[:, o], y, s, TOL[tnsk.PREC_FP32], f"{spec.name} entry {o} (batch)")
    X = rounded(chain, torch.float32)
    y, s = oracle.m1_estimate(X, chain.edges, chain.open, m=p1.m, reps=p1.reps, seed=p1.seed)
    assert_parity(pers[2].cpu().numpy(), y, s, TOL[tnsk.PREC_FP32], "method 1 beside them")
    with pytest.raises(tnsk.TnskError):
        ctx.plan([nets[0]], [p], [outs[0]])


def test_method2_open_legs_limits(ctx):
    """More than 2^16 output entries in one call, or an empty output, are refused with
    TNSK_ERR_UNSUPPORTED (each entry is a full estimate of its own)."""
    rng = np.random.default_rng(3)
    big = W.NetSpec([rng.standard_normal((300, 5)).astype(np.float32), rng.standard_normal((5, 300)).astype(np.float32)],
                    [(1, 2)], [0, 3], "90000 entries")
    empty = W.NetSpec([np.zeros((0, 5), dtype=np.float32), rng.standard_normal((5, 4)).astype(np.float32)],
                      [(1, 2)], [0, 3], "empty output")
    p = tnsk.Params(m=64, reps=2, seed=1, method=tnsk.ACYCLIC)
    for spec in (big, empty):
        net = gpu_network(spec, torch.float32)
        out = torch.zeros(max(1, 300 * 300), dtype=torch.float64, device="cuda")
        with pytest.raises(tnsk.TnskError):
            ctx.estimate(net, p, out)
