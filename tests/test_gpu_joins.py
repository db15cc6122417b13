"""Join-size estimation (Sec. 5.1): the frequency tensors of a query's relations fed
to a turnstile stream as updates, the three-way join class given as a hyperedge (the
library appends its copy tensor, WLOG 1), against the FP64 oracle's estimate on the
dense tensors with its own copy tensor and the same hashes."""
import numpy as np
import pytest

import oracle
from oracle.normalize import copy_tensors
from gpu_common import TOL, assert_parity
from paper_2603_07387_gb300 import joins, tnsk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tnsk.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def _zipf(rng, n, size, a=1.3):
    return np.minimum(rng.zipf(a, size) - 1, n - 1)


def test_paper_query_with_a_three_way_join_class(ctx):
    # R1.1 = R2.2, R3.4 = R2.2, R4.5 = R2.3 (the paper's example query; 0-based columns)
    rng = np.random.default_rng(41)
    R1 = _zipf(rng, 40, (900, 1))
    R2 = np.stack([_zipf(rng, 40, 1200), _zipf(rng, 30, 1200)], 1)
    R3 = _zipf(rng, 40, (700, 1))
    R4 = _zipf(rng, 30, (500, 1))
    jn = joins.join_network([R1, R2, R3, R4], [((0, 0), (1, 0)), ((2, 0), (1, 0)), ((3, 0), (1, 1))])
    assert len(jn.shapes) == 4 and len(jn.edges) == 3  # mode 1 (R2's first column) in two contractions
    p = tnsk.Params(m=1024, reps=16, seed=77, method=tnsk.GENERAL)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    per = torch.zeros((p.reps, 1), dtype=torch.float64, device="cuda")
    st = ctx.stream(tnsk.Network([tnsk.Zeros(*sh) for sh in jn.shapes], jn.edges, []), p, out, per)
    k = np.concatenate([np.full(u.size, i, dtype=np.int32) for i, u in enumerate(jn.updates)])
    flat = np.concatenate(jn.updates)
    st.update(torch.as_tensor(k, device="cuda"), torch.as_tensor(flat, device="cuda"),
              torch.ones(flat.size, dtype=torch.float64, device="cuda"))
    st.estimate()
    ctx.sync()
    X, E, _ = copy_tensors(joins.exact_dense_tensors(jn), jn.edges)
    assert len(X) == 5 and X[4].ndim == 3  # the copy tensor of the three-way class
    y, s = oracle.m1_estimate(X, E, [], m=p.m, reps=p.reps, seed=p.seed)
    assert_parity(per.cpu().numpy(), y, s, TOL[p.prec], "join")
    # the dense contraction is the join size
    exact = float(np.asarray(oracle.tc_einsum(X, E, [])))
    f1, f3 = np.bincount(R1[:, 0], minlength=40), np.bincount(R3[:, 0], minlength=40)
    f4 = np.bincount(R4[:, 0], minlength=30)
    want = sum(f1[a] * f3[a] * f4[b] for a, b in R2)
    assert exact == want
    st.close()
