"""tnsk_estimate_static: the method-1 estimate for callers that cannot allocate
device memory (inside a stream capture they do not own, or under a host
application that owns every allocation). It keeps all scratch in the library's
fixed 16 MiB device array. Checked through the C ABI against tnsk_estimate on two
calls in a row, within the parity tolerance of the other GPU tests (1e-5 of the
oracle's cancellation-aware scale, FP32 path).

This file is collected last on purpose, so a failure here comes after every
other test has run."""
import ctypes

import numpy as np
import pytest

from paper_2603_07387_gb300 import tnsk
from paper_2603_07387_gb300 import workloads as W

from gpu_common import TOL, gpu_network, oracle_estimate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _specs():
    rng = np.random.default_rng(31)
    return [W.triangle(64), W.random_network(rng, p_range=(4, 6), dim_range=(2, 6), open_dim_range=(2, 4)),
            W.grid(3, 3, 4, seed=5)]


def _call_static(lib, net, params, out, per, stream):
    nh = tnsk._NetHolder(net)
    pr = tnsk._params(params)
    return lib.tnsk_estimate_static(ctypes.byref(nh.c), ctypes.byref(pr), ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(per.data_ptr()), ctypes.c_void_p(stream))


def test_static_scratch_estimate_matches_tnsk_estimate_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = tnsk.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    ctx = tnsk.Context(0, stream)
    try:
        for spec in _specs():
            params = tnsk.Params(m=256, reps=16, groups=4, seed=W.HASH_SEED)
            net = gpu_network(spec, torch.float32)
            dims = [d for x in spec.tensors for d in np.shape(x)]
            O = int(np.prod([dims[g] for g in spec.open])) if spec.open else 1
            ref_out = torch.zeros(max(O, 1), dtype=torch.float64, device="cuda")
            ref_per = torch.zeros((params.reps, max(O, 1)), dtype=torch.float64, device="cuda")
            ctx.estimate(net, params, ref_out, ref_per)
            ctx.sync()
            _, scale = oracle_estimate(spec, params, torch.float32)
            for call in range(2):
                out = torch.full((max(O, 1),), np.nan, dtype=torch.float64, device="cuda")
                per = torch.full((params.reps, max(O, 1)), np.nan, dtype=torch.float64, device="cuda")
                st = _call_static(lib, net, params, out, per, stream)
                assert st == 0, f"call {call}: status {st}"
                torch.cuda.synchronize()
                got = per.cpu().numpy()[:, :O]
                want = ref_per.cpu().numpy()[:, :O]
                assert np.all(np.abs(got - want) <= TOL[tnsk.PREC_FP32] * scale), (spec.name, call)
                # the combination of the same per-rep values is identical
                g_out = out.cpu().numpy()[:O]
                r_out = ref_out.cpu().numpy()[:O]
                assert np.all(np.abs(g_out - r_out) <= TOL[tnsk.PREC_FP32] * scale.max(axis=0)), (spec.name, call)
    finally:
        ctx.close()


def test_static_scratch_rejects_oversize_and_other_methods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = tnsk.load_library()
    stream = torch.cuda.current_stream().cuda_stream
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
