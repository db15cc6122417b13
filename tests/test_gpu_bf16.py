"""TNSK_PREC_BF16 against the oracle, and the cyclic 4 x 4 grid of bond 8 at full size.

BF16 path (tensors stored as BF16): method 2's sketched product runs on the BF16
tensor cores (X as stored, V as three BF16 parts, FP32 accumulation), so the result
is FP32 arithmetic on the BF16 values. Checked per repetition against the oracle on
the BF16-rounded inputs at the FP32 tolerance (1e-5 of the oracle's
cancellation-aware scale: only accumulation order and V's 2^-24 split differ), and
against the oracle on the original inputs at 1e-2 (the BF16 tolerance: BF16 keeps 8
significant bits, so every entry moves by at most 2^-9 of itself).

The grid (16 tensors, interior order 4, U(0,1) entries, t = 24 contractions) runs
method 1 at m = 2^10 and 2^16 (the transform's register, block and two-pass forms
are all covered by the other tests; 2^16 is the largest m), FP32 and BF16 storage."""
import numpy as np
import pytest

import oracle
from paper_2603_07387_gb300 import tnsk
from paper_2603_07387_gb300 import workloads as W

from gpu_common import TOL, assert_parity, gpu_estimate, oracle_estimate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BF16_TOL = 1e-2


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tnsk.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def _chain(rng, dims, name):
    """Vector - matrices - vector chain with the given bond dims (parent modes first when
    rooted at the leading vector, the default root: the tensor with fewest entries)."""
    X = [rng.standard_normal(dims[0])]
    for a, b in zip(dims[:-1], dims[1:]):
        X.append(rng.standard_normal((a, b)) / np.sqrt(a))
    X.append(rng.standard_normal(dims[-1]))
    edges, g = [], 0
    for x in X[:-1]:
        g += x.ndim
        edges.append((g - 1, g))
    return W.NetSpec(X, edges, [], name)


def _bf16_specs():
    rng = np.random.default_rng(5)
    A, B = W.tt_cores(sites=4, bond=8, phys=4, seed=3)
    return [W.tt_chain(A, B),                                   # 64 x 64 sites: one tile, one chunk
            _chain(rng, [200, 136, 72, 264], "ragged"),          # rows and columns off the tile and chunk sizes
            _chain(rng, [256, 1024, 512], "wide")]               # several chunks (and K splits)


@pytest.mark.parametrize("reps", [8, 70])
def test_bf16_method2_parity(ctx, reps):
    for spec in _bf16_specs():
        p = tnsk.Params(m=256, reps=reps, seed=41, method=tnsk.ACYCLIC, prec=tnsk.PREC_BF16)
        out, per = gpu_estimate(ctx, spec, p, torch.bfloat16)
        y, s = oracle_estimate(spec, p, torch.bfloat16)  # the oracle on the BF16-rounded inputs
        assert_parity(per, y, s, TOL[tnsk.PREC_FP32], f"{spec.name} vs BF16 inputs")
        y64, s64 = oracle_estimate(spec, p, torch.float64)  # the oracle on the original inputs
        assert_parity(per, y64, s64, BF16_TOL, f"{spec.name} vs FP64 inputs")
        # the combination of the same per-rep values
        assert np.allclose(out, oracle.combine(per, 1), rtol=1e-14, atol=0)


def test_bf16_method2_same_as_fp32_mode_on_bf16_values(ctx):
    """The BF16 kernel and the FP32 path (TF32 split) on the same BF16 tensors agree to
    the FP32 tolerance."""
    spec = _bf16_specs()[2]
    pb = tnsk.Params(m=512, reps=16, seed=9, method=tnsk.ACYCLIC, prec=tnsk.PREC_BF16)
    pf = tnsk.Params(m=512, reps=16, seed=9, method=tnsk.ACYCLIC, prec=tnsk.PREC_FP32)
    _, per_b = gpu_estimate(ctx, spec, pb, torch.bfloat16)
    _, per_f = gpu_estimate(ctx, spec, pf, torch.bfloat16)
    _, s = oracle_estimate(spec, pf, torch.bfloat16)
    assert np.all(np.abs(per_b - per_f) <= 2 * TOL[tnsk.PREC_FP32] * s)


@pytest.mark.parametrize("m", [1 << 10, 1 << 16])
def test_grid_4x4_bond8_full_size(ctx, m):
    """The cyclic 4 x 4 grid of bond 8 (U(0,1), 20,736 entries), method 1, FP32 and BF16
    storage, against the oracle on the same (rounded) inputs at 1e-5 and, for BF16, on
    the FP32 inputs at 1e-2."""
    spec = W.grid(4, 4, 8)
    reps = 4
    for prec, tdt in ((tnsk.PREC_FP32, torch.float32), (tnsk.PREC_BF16, torch.bfloat16)):
        p = tnsk.Params(m=m, reps=reps, seed=W.HASH_SEED, prec=prec)
        out, per = gpu_estimate(ctx, spec, p, tdt)
        y, s = oracle_estimate(spec, p, tdt)
        assert_parity(per, y, s, TOL[tnsk.PREC_FP32], f"grid m={m} prec={prec}")
        if prec == tnsk.PREC_BF16:
            y32, s32 = oracle_estimate(spec, p, torch.float32)
            assert_parity(per, y32, s32, BF16_TOL, f"grid m={m} BF16 vs FP32 inputs")


def test_bf16_precision_fp32_tensors_take_the_fp32_path(ctx):
    """Tensors of other dtypes in BF16 mode take the FP32 path (same results as FP32
    mode within the FP32 tolerance)."""
    spec = _bf16_specs()[1]
    pb = tnsk.Params(m=256, reps=8, seed=12, method=tnsk.ACYCLIC, prec=tnsk.PREC_BF16)
    _, per = gpu_estimate(ctx, spec, pb, torch.float32)
    y, s = oracle_estimate(spec, pb, torch.float32)
    assert_parity(per, y, s, TOL[tnsk.PREC_FP32], "FP32 tensors in BF16 mode")
