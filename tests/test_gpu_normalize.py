"""GPU parity of the acyclic method on networks that need the WLOG 2 / WLOG 3
rewrite of Sec. 4.1 (contractions inside one tensor, several contractions between
two tensors): libtnsk rewrites them itself before method 2; the oracle rewrites the
same dtype-rounded tensors with its own numpy code (oracle.normalize) and runs its
method 2 on the result with the same seeds. Per-rep estimates are compared with
the cancellation-aware tolerance of the other parity tests."""
import numpy as np
import pytest

import oracle
from oracle.normalize import normalize
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


def _mixed(seed=0, scale=(6, 5, 7, 4, 3)):
    """A(6,5,7,7) joins B(5,6,4) twice, listed (A1,B0) before (A0,B1): A's merged mode
    is (i1, i0) and needs a transpose, B's is (i0, i1) and only a reshape; A's modes 2,
    3 and C's modes 1, 2 are traced; B-C is a single contraction. The rewrite is the
    chain A'(30) - B'(30,4) - C'(4)."""
    a, b, c, d, e = scale
    rng = np.random.default_rng(seed)
    X = [rng.standard_normal((a, b, c, c)), rng.standard_normal((b, a, d)), rng.standard_normal((d, e, e))]
    edges = [(1, 4), (0, 5), (2, 3), (6, 7), (8, 9)]
    return W.NetSpec(X, edges, [], "wlog-mixed")


def _oracle_normalized(spec, params, tdt):
    X = rounded(spec, tdt)
    T, E, _ = normalize(X, spec.edges)
    root = params.root
    if root < 0:
        root = int(np.argmin([t.size for t in T]))
    return oracle.m2_estimate(T, E, m=params.m, reps=params.reps, seed=params.seed, root=root)


@pytest.mark.parametrize("prec,dtype", [(tnsk.PREC_FP32, "float32"), (tnsk.PREC_FP64, "float64"),
                                        (tnsk.PREC_FP32, "bfloat16")])
@pytest.mark.parametrize("root", [-1, 0, 1, 2])
def test_traces_and_merged_contractions(ctx, prec, dtype, root):
    spec = _mixed(seed=1)
    tdt = getattr(torch, dtype)
    p = tnsk.Params(m=64, reps=7, seed=31, method=tnsk.ACYCLIC, root=root, prec=prec)
    out, per = gpu_estimate(ctx, spec, p, tdt)
    y, s = _oracle_normalized(spec, p, tdt)
    assert_parity(per, y[:, None], s[:, None], TOL[prec], f"wlog mixed {dtype} root={root}")


def test_rewrite_at_tile_sizes(ctx):
    """Sizes past the tensor-core tiles: A(24,40,9,9) and B(40,24,130) joined twice
    (A's merged mode transposed, 960 wide), B-C on 130, C(130,5,5) traced."""
    spec = _mixed(seed=2, scale=(24, 40, 9, 130, 5))
    p = tnsk.Params(m=256, reps=70, seed=5, method=tnsk.ACYCLIC, root=0)
    out, per = gpu_estimate(ctx, spec, p, torch.float32)
    y, s = _oracle_normalized(spec, p, torch.float32)
    assert_parity(per, y[:, None], s[:, None], TOL[p.prec], "wlog tiles")


def test_paper_examples_and_plans(ctx):
    """tr(M) alone (the whole network traced: exact for every rep), the WLOG 3 example
    vec(A) . vec(B), and a plan of both (graph replays) equal to single estimates."""
    rng = np.random.default_rng(9)
    M = rng.standard_normal((33, 33))
    tr = W.NetSpec([M], [(1, 0)], [], "trace")
    p = tnsk.Params(m=16, reps=3, seed=2, method=tnsk.ACYCLIC, prec=tnsk.PREC_FP64)
    _, per = gpu_estimate(ctx, tr, p, torch.float64)
    assert np.allclose(per, np.trace(M), rtol=1e-12)
    A, B = rng.standard_normal((12, 20)), rng.standard_normal((12, 20))
    ab = W.NetSpec([A, B], [(0, 2), (1, 3)], [], "vec-inner")
    p2 = tnsk.Params(m=512, reps=9, seed=3, method=tnsk.ACYCLIC, root=1)
    _, per2 = gpu_estimate(ctx, ab, p2, torch.float32)
    y, s = _oracle_normalized(ab, p2, torch.float32)
    assert_parity(per2, y[:, None], s[:, None], TOL[p2.prec], "vec-inner")
    # plan: the mixed network and the WLOG 3 example in one batch with a plain tree
    tree = W.NetSpec([rng.standard_normal(8), rng.standard_normal((8, 5)), rng.standard_normal(5)],
                     [(0, 1), (2, 3)], [], "plain")
    mixed = _mixed(seed=3)
    specs = [mixed, ab, tree]
    params = [tnsk.Params(m=128, reps=6, seed=40 + i, method=tnsk.ACYCLIC, root=i) for i in range(3)]
    nets = [gpu_network(s, torch.float32) for s in specs]
    outs = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in specs]
    pers = [torch.zeros((6, 1), dtype=torch.float64, device="cuda") for _ in specs]
    plan = ctx.plan(nets, params, outs, pers)
    for _ in range(3):
        for t in pers:
            t.zero_()
        plan.run()
        ctx.sync()
        for s, pr, pe in zip(specs, params, pers):
            y, sc = _oracle_normalized(s, pr, torch.float32)
            assert_parity(pe.cpu().numpy(), y[:, None], sc[:, None], TOL[pr.prec], f"plan {s.name}")
    plan.close()
    # a batch through tnsk_estimate_batch gives the same
    bouts = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in specs]
    bpers = [torch.zeros((6, 1), dtype=torch.float64, device="cuda") for _ in specs]
    ctx.estimate_batch(nets, params, bouts, bpers)
    ctx.sync()
    for s, pr, pe in zip(specs, params, bpers):
        y, sc = _oracle_normalized(s, pr, torch.float32)
        assert_parity(pe.cpu().numpy(), y[:, None], sc[:, None], TOL[pr.prec], f"batch {s.name}")


def test_rewrite_errors(ctx):
    """A cycle through three tensors stays a cycle after merging (TNSK_ERR_CYCLIC); a
    grouped (rung) tensor that would need a trace is refused (TNSK_ERR_UNSUPPORTED)."""
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    A = [np.ones((3, 3, 3)), np.ones((3, 3, 3)), np.ones((3, 3))]  # modes 0-2, 3-5, 6-7
    # A-B twice, B-C, C-A: after the merge a triangle
    spec = W.NetSpec(A, [(0, 3), (1, 4), (5, 6), (7, 2)], [])
    with pytest.raises(tnsk.TnskError) as e:
        ctx.estimate(gpu_network(spec, torch.float32), tnsk.Params(m=8, reps=2, method=tnsk.ACYCLIC), out)
    assert e.value.status == -2
    a = torch.ones((2, 3, 2), device="cuda")
    rung = tnsk.Rung(a, a)  # [4, 4]
    with pytest.raises(tnsk.TnskError) as e:
        ctx.estimate(tnsk.Network([rung], [(0, 1)], []), tnsk.Params(m=8, reps=2, method=tnsk.ACYCLIC), out)
    assert e.value.status == -3
    ctx.sync()
