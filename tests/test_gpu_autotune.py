"""The scatter-schedule autotuner (tnsk_autotune) and scheduled plans against the oracle.

A schedule only regroups row a2's work (how many reps one work item sketches in one
pass over its entries, how many entries one item takes), so every schedule must give
the oracle's per-rep estimates at the FP32 tolerance. Checked on a batch that fills
every kind of scatter list (orders 2..7, open legs, four-entry and single-entry loads,
privatised and global bins, tensors of several chunks): a forced schedule at the
extremes of the candidate grid, and the schedule the autotuner picks, whose summed
scatter time is at most the default's by construction."""
import numpy as np
import pytest

from paper_2603_07387_gb300 import tnsk
from paper_2603_07387_gb300 import workloads as W

from gpu_common import TOL, assert_parity, gpu_network, oracle_estimate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tnsk.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def _batch():
    rng = np.random.default_rng(404)
    specs = [W.random_network(rng, p_range=(4, 7), dim_range=(2, 9), open_dim_range=(2, 5)) for _ in range(10)]
    A, B = W.tt_cores(sites=6, bond=16, phys=4, seed=8)
    specs.append(W.tt_ladder(A, B))  # order-3 cores of 1024 entries, four-entry loads
    specs.append(W.grid(3, 3, 6, seed=4))
    big = rng.standard_normal((40, 36, 30))  # 43200 entries: several chunks at m = 256
    specs.append(W.NetSpec([big, rng.standard_normal((30, 40)), rng.standard_normal(36)], [(0, 4), (2, 3), (1, 5)],
                           [], "big-chunks"))
    ms = [256, 1024]
    params = [tnsk.Params(m=ms[i % 2], reps=12, seed=600 + i) for i in range(len(specs))]
    return specs, params


def _run(ctx, specs, params, schedule):
    nets = [gpu_network(s, torch.float32) for s in specs]
    outs, pers, Os = [], [], []
    for s, p in zip(specs, params):
        dims = [d for x in s.tensors for d in np.shape(x)]
        O = int(np.prod([dims[g] for g in s.open])) if s.open else 1
        Os.append(O)
        outs.append(torch.zeros(max(O, 1), dtype=torch.float64, device="cuda"))
        pers.append(torch.zeros((p.reps, max(O, 1)), dtype=torch.float64, device="cuda"))
    plan = ctx.plan(nets, params, outs, pers, schedule=schedule)
    plan.run()
    plan.run()
    ctx.sync()
    plan.close()
    return [p.cpu().numpy()[:, :O] for p, O in zip(pers, Os)]


def _check(specs, params, pers, what):
    for s, p, per in zip(specs, params, pers):
        y, sc = oracle_estimate(s, p, torch.float32)
        assert_parity(per, y, sc, TOL[p.prec], f"{what}: {s.name} m={p.m}")


def test_forced_schedules_match_oracle(ctx):
    specs, params = _batch()
    for cap, scale in ((8, 4), (32, 1), (16, 2)):
        sched = tnsk.Schedule()
        for l in range(tnsk.SCATTER_LISTS):
            sched.rep_cap[l] = cap
            sched.chunk_scale[l] = scale
        _check(specs, params, _run(ctx, specs, params, sched), f"rep_cap {cap} chunk_scale {scale}")


def test_autotuned_schedule(ctx):
    specs, params = _batch()
    nets = [gpu_network(s, torch.float32) for s in specs]
    sched, ms_def, ms_tuned = ctx.autotune(nets, params, trials=2)
    assert ms_def > 0 and 0 < ms_tuned <= ms_def
    for l in range(tnsk.SCATTER_LISTS):
        assert sched.rep_cap[l] in (0, 8, 16, 32)
        assert sched.chunk_scale[l] in (0, 1, 2, 4)
    _check(specs, params, _run(ctx, specs, params, sched), "autotuned")


def test_autotune_arguments(ctx):
    specs, params = _batch()
    nets = [gpu_network(s, torch.float32) for s in specs[:2]]
    with pytest.raises(tnsk.TnskError) as e:
        ctx.autotune(nets, params[:2], trials=0)
    assert e.value.status == -1
