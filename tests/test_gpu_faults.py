"""Failure detection on the GPU without a fault: a test-only switch
(tnsk_debug_inject) makes the next method-2 tensor-core product's TMA producers
issue no loads. Its consumers' mbarrier waits are bounded (polls and about 2^31 SM
cycles), so they run out, record TNSK_ERR_TIMEOUT for tnsk_sync, and every warp still
releases its tensor memory; the next call on the same ctx runs normally and matches
the oracle."""
import numpy as np
import pytest

from paper_2603_07387_gb300 import tnsk

from gpu_common import TOL, assert_parity, gpu_estimate, oracle_estimate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _chain(dtype_seed=3):
    from paper_2603_07387_gb300 import workloads as W

    rng = np.random.default_rng(dtype_seed)
    X = [rng.standard_normal(256), rng.standard_normal((256, 512)) / 16.0, rng.standard_normal(512)]
    return W.NetSpec(X, [(0, 1), (2, 3)], [], "chain")


@pytest.mark.parametrize("prec,tdt", [(tnsk.PREC_FP32, "float32"), (tnsk.PREC_BF16, "bfloat16")])
def test_injected_wait_reports_timeout_and_ctx_recovers(prec, tdt):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dt = getattr(torch, tdt)
    ctx = tnsk.Context(0, torch.cuda.current_stream().cuda_stream)
    try:
        spec = _chain()
        p = tnsk.Params(m=256, reps=8, seed=17, method=tnsk.ACYCLIC, prec=prec)
        ctx.debug_inject(1)
        with pytest.raises(tnsk.TnskError) as e:
            gpu_estimate(ctx, spec, p, dt)
        assert e.value.status == -6  # TNSK_ERR_TIMEOUT
        # the switch was one-shot and the ctx is intact: a normal call matches the oracle
        _, per = gpu_estimate(ctx, spec, p, dt)
        y, s = oracle_estimate(spec, p, dt)
        assert_parity(per, y, s, TOL[tnsk.PREC_FP32], "after the injected timeout")
    finally:
        ctx.close()


def test_inject_rejects_unknown_values():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = tnsk.Context(0, torch.cuda.current_stream().cuda_stream)
    try:
        with pytest.raises(tnsk.TnskError):
            ctx.debug_inject(7)
    finally:
        ctx.close()
