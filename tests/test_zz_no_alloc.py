"""tnsk_estimate_static: the method-1 estimate for callers that cannot allocate
device memory (a host application that owns every allocation, or a deployment
where device memory must not grow after start-up). It keeps all scratch in the
library's fixed 16 MiB device array. Checked through the C ABI against
tnsk_estimate and against the oracle on two calls in a row, within the parity
tolerance of the other GPU tests (1e-5 of the oracle's cancellation-aware scale,
FP32 path); also without per-rep output, after a larger call (nothing stale may
leak into a smaller one), and on a hyperedge network (WLOG 1 copy tensors).

This file is collected last on purpose, so a failure here comes after every
other test has run."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle.normalize import copy_tensors
from paper_2603_07387_gb300 import tnsk
from paper_2603_07387_gb300 import workloads as W

from gpu_common import TOL, assert_parity, gpu_network, oracle_estimate, rounded

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _specs():
    rng = np.random.default_rng(31)
    return [W.triangle(64), W.random_network(rng, p_range=(4, 6), dim_range=(2, 6), open_dim_range=(2, 4)),
            W.grid(3, 3, 4, seed=5)]


def _call_static(lib, net, params, out, per, stream):
    nh = tnsk._NetHolder(net)
    pr = tnsk._params(params)
    per_ptr = ctypes.c_void_p(per.data_ptr()) if per is not None else ctypes.c_void_p(None)
    return lib.tnsk_estimate_static(ctypes.byref(nh.c), ctypes.byref(pr), ctypes.c_void_p(out.data_ptr()), per_ptr,
                                    ctypes.c_void_p(stream))


def _outsize(spec):
    dims = [d for x in spec.tensors for d in np.shape(x)]
    return int(np.prod([dims[g] for g in spec.open])) if spec.open else 1


def _reference(ctx, net, params, O):
    ref_out = torch.zeros(max(O, 1), dtype=torch.float64, device="cuda")
    ref_per = torch.zeros((params.reps, max(O, 1)), dtype=torch.float64, device="cuda")
    ctx.estimate(net, params, ref_out, ref_per)
    ctx.sync()
    return ref_out.cpu().numpy()[:O], ref_per.cpu().numpy()[:, :O]


def _static(lib, net, params, O, stream, with_per=True):
    out = torch.full((max(O, 1),), np.nan, dtype=torch.float64, device="cuda")
    per = torch.full((params.reps, max(O, 1)), np.nan, dtype=torch.float64, device="cuda") if with_per else None
    st = _call_static(lib, net, params, out, per, stream)
    assert st == 0, f"status {st}"
    torch.cuda.synchronize()
    return out.cpu().numpy()[:O], (per.cpu().numpy()[:, :O] if with_per else None)


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = tnsk.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    ctx = tnsk.Context(0, stream)
    yield lib, stream, ctx
    ctx.close()


def test_static_scratch_estimate_matches_tnsk_estimate_twice(env):
    lib, stream, ctx = env
    tol = TOL[tnsk.PREC_FP32]
    for spec in _specs():
        params = tnsk.Params(m=256, reps=16, groups=4, seed=W.HASH_SEED)
        net = gpu_network(spec, torch.float32)
        O = _outsize(spec)
        r_out, r_per = _reference(ctx, net, params, O)
        y, scale = oracle_estimate(spec, params, torch.float32)
        for call in range(2):
            g_out, g_per = _static(lib, net, params, O, stream)
            assert np.all(np.abs(g_per - r_per) <= tol * scale), (spec.name, call)
            assert_parity(g_per, y, scale, tol, f"{spec.name} call {call} vs oracle")
            # the combination of the same per-rep values agrees
            assert np.all(np.abs(g_out - r_out) <= tol * scale.max(axis=0)), (spec.name, call)
            o_out = oracle.combine(y, params.groups)
            assert np.all(np.abs(g_out - o_out) <= tol * scale.max(axis=0)), (spec.name, call)


def test_static_scratch_without_per_rep_and_after_a_larger_call(env):
    lib, stream, ctx = env
    tol = TOL[tnsk.PREC_FP32]
    small = W.random_network(np.random.default_rng(8), p_range=(4, 5), dim_range=(2, 5), open_dim_range=(2, 3))
    big = W.grid(3, 3, 4, seed=9)
    p_small = tnsk.Params(m=64, reps=8, seed=3)
    p_big = tnsk.Params(m=4096, reps=32, seed=4)  # ~4.5 MiB of sketches, more than the small call needs
    n_small, n_big = gpu_network(small, torch.float32), gpu_network(big, torch.float32)
    O = _outsize(small)
    y, scale = oracle_estimate(small, p_small, torch.float32)
    r_out, r_per = _reference(ctx, n_small, p_small, O)
    for _ in range(2):
        _static(lib, n_big, p_big, 1, stream)
        g_out, g_per = _static(lib, n_small, p_small, O, stream)
        assert_parity(g_per, y, scale, tol, "small call after a large one")
        assert np.all(np.abs(g_out - r_out) <= tol * scale.max(axis=0))
        _static(lib, n_big, p_big, 1, stream)
        g_out, _ = _static(lib, n_small, p_small, O, stream, with_per=False)
        assert np.all(np.abs(g_out - r_out) <= tol * scale.max(axis=0)), "per_rep = NULL"


def test_static_scratch_hyperedges(env):
    """A mode in two contractions (the paper's sum_i a(i) b(i) c(i)): WLOG 1's copy
    tensor, sketched from its nonzeros, as in tnsk_estimate."""
    lib, stream, ctx = env
    rng = np.random.default_rng(44)
    spec = W.NetSpec([rng.standard_normal(9) for _ in range(3)], [(0, 1), (1, 2)], [], "abc")
    params = tnsk.Params(m=64, reps=6, seed=61)
    T, E, Op = copy_tensors(rounded(spec, torch.float32), spec.edges, spec.open)
    y, s = oracle.m1_estimate(T, E, Op, m=params.m, reps=params.reps, seed=params.seed)
    for _ in range(2):
        _, g_per = _static(lib, gpu_network(spec, torch.float32), params, 1, stream)
        assert_parity(g_per, y, s, TOL[tnsk.PREC_FP32], "static hyperedge")


def test_static_scratch_rejects_oversize_and_other_methods(env):
    lib, stream, _ = env
    spec = W.triangle(8)
    net = gpu_network(spec, torch.float32)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # 4096 reps x 3 tensors x m = 4096 FP32 sketches = 192 MiB of scratch > 16 MiB
    big = tnsk.Params(m=4096, reps=4096, seed=1)
    per = torch.zeros((big.reps, 1), dtype=torch.float64, device="cuda")
    assert _call_static(lib, net, big, out, per, stream) == -3
    acyc = tnsk.Params(m=64, reps=4, seed=1, method=tnsk.ACYCLIC)
    assert _call_static(lib, net, acyc, out, per, stream) == -3
    torch.cuda.synchronize()
