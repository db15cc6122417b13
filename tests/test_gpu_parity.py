"""GPU parity: libtnsk (through the C ABI) against the FP64 oracle, same seeds.

Rows covered: a1 tables (bit-exact), a2 method-1 sketches (per bin), a3+a4
method-1 estimates (per rep), a5-a8 method-2 estimates (per rep), a9 combination.
Tolerance: |gpu - oracle| <= tol * S with S the oracle's cancellation-aware scale
(tol 1e-5 for the FP32 path, 1e-10 for the FP64 path)."""
import numpy as np
import pytest

import oracle
from paper_2603_07387_gb300 import tnsk
from paper_2603_07387_gb300 import workloads as W

from gpu_common import sketch_tol, TOL, assert_parity, gpu_estimate, gpu_network, oracle_estimate, rounded

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = tnsk.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


# ---------------------------------------------------------------- a1 tables
@pytest.mark.parametrize("seed,rep,tid,n,m", [
    (0, 0, 1 << 56, 1000, 1024), (0x7E57, 7, (4 << 56) | (3 << 24) | (2 << 16) | 5, 4096, 4096),
    (2**64 - 1, 65535, (2 << 56) | 9, 33, 1), (5, 1, (3 << 56) | 1, 100_000, 65536), (1, 2, 3, 0, 8)])
def test_count_sketch_bit_exact(ctx, seed, rep, tid, n, m):
    bins = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    signs = torch.zeros(max(n, 1), dtype=torch.int8, device="cuda")
    ctx.count_sketch(seed, rep, tid, n, m, bins, signs)
    ctx.sync()
    ob, os_ = oracle.count_sketch(seed, rep, tid, n, m)
    assert np.array_equal(bins.cpu().numpy()[:n], ob)
    assert np.array_equal(signs.cpu().numpy()[:n], os_)


# ---------------------------------------------------------------- a2 sketches
def _small_specs():
    rng = np.random.default_rng(11)
    specs = [W.triangle(5, seed=1)]
    specs.append(W.NetSpec([rng.standard_normal((3, 4, 2)), rng.standard_normal((4, 5)), rng.standard_normal((5, 3))],
                           [(1, 3), (4, 5), (6, 0)], [2], "open1"))
    specs.append(W.NetSpec([rng.standard_normal((3, 2, 3)), rng.standard_normal(2)], [(0, 2), (1, 3)], [],
                           "selftrace"))
    specs.append(W.random_network(np.random.default_rng(3), p_range=(4, 6), dim_range=(2, 5), open_dim_range=(2, 3)))
    specs.append(W.grid(2, 3, 3, seed=4))
    return specs


@pytest.mark.parametrize("prec,m", [(tnsk.PREC_FP64, 8), (tnsk.PREC_FP64, 1), (tnsk.PREC_FP32, 64),
                                    (tnsk.PREC_FP32, 2), (tnsk.PREC_FP32, 1024)])
def test_method1_sketch_per_bin(ctx, prec, m):
    R, seed = 5, 0x7E57
    for spec in _small_specs():
        tdt = torch.float64 if prec == tnsk.PREC_FP64 else torch.float32
        net = gpu_network(spec, tdt)
        X = rounded(spec, tdt)
        bins, signs = oracle.m1_tables(X, spec.edges, spec.open, seed=seed, reps=R, m=m)
        want = oracle.m1_sketch(X, spec.edges, spec.open, m, bins, signs)
        scale = oracle.m1_sketch(X, spec.edges, spec.open, m, bins, signs, abs_mode=True)
        x = torch.zeros(want.shape, dtype=tdt, device="cuda")
        ctx.m1_sketch(net, tnsk.Params(m=m, reps=R, seed=seed, prec=prec), x)
        ctx.sync()
        got = x.double().cpu().numpy()
        bound = sketch_tol(X, spec.edges, spec.open, m, bins, signs, prec)
        assert np.all(np.abs(got - want) <= bound), spec.name


# ---------------------------------------------------------------- a3 + a4 method 1
@pytest.mark.parametrize("prec", [tnsk.PREC_FP32, tnsk.PREC_FP64])
@pytest.mark.parametrize("m", [1, 2, 16, 256, 4096])
def test_method1_estimate_small(ctx, prec, m):
    tdt = torch.float64 if prec == tnsk.PREC_FP64 else torch.float32
    for spec in _small_specs():
        p = tnsk.Params(m=m, reps=6, groups=3, seed=99, prec=prec)
        out, per = gpu_estimate(ctx, spec, p, tdt)
        y, s = oracle_estimate(spec, p, tdt)
        assert_parity(per, y, s, TOL[prec], f"{spec.name} m={m}")
        assert np.allclose(out, oracle.combine(per, 3), rtol=1e-14, atol=0)


@pytest.mark.parametrize("prec", [tnsk.PREC_FP32, tnsk.PREC_FP64])
def test_method1_large_tables_from_global_memory(ctx, prec):
    """Modes above 2048 indices: the scatter stages only the index ranges a chunk touches
    (tr(ABC) with long inner modes, a chain with an open leg), or, where even those do
    not fit next to the bins (a 20000-index last mode at m = 2^14), reads the table
    words from global memory with the complement applied on the fly; against the
    oracle."""
    rng = np.random.default_rng(17)
    tdt = torch.float64 if prec == tnsk.PREC_FP64 else torch.float32
    A, B, C = rng.standard_normal((3000, 5)), rng.standard_normal((5, 2100)), rng.standard_normal((2100, 3000))
    tri = W.NetSpec([A, B, C], [(1, 2), (3, 4), (5, 0)], [], "long-modes")
    chain = W.NetSpec([rng.standard_normal((2500, 3)), rng.standard_normal((2500, 4))], [(0, 2)], [1, 3], "open")
    wide = W.NetSpec([rng.standard_normal((3, 20000)), rng.standard_normal((20000, 3))], [(1, 2), (3, 0)], [], "wide")
    for spec, m in [(tri, 256), (tri, 4096), (chain, 64), (wide, 1 << 14)]:
        p = tnsk.Params(m=m, reps=9, seed=21, prec=prec)
        out, per = gpu_estimate(ctx, spec, p, tdt)
        y, s = oracle_estimate(spec, p, tdt)
        assert_parity(per, y, s, TOL[prec], f"{spec.name} m={m}")


def test_method1_triangle_full_size(ctx):
    """tr(ABC) of three 64x64 FP64 N(0,1) matrices, m = 256, 16 reps."""
    spec = W.triangle(64)
    for prec in (tnsk.PREC_FP32, tnsk.PREC_FP64):
        p = tnsk.Params(m=256, reps=16, seed=W.HASH_SEED, prec=prec)
        out, per = gpu_estimate(ctx, spec, p, torch.float64)
        y, s = oracle_estimate(spec, p, torch.float64)
        assert_parity(per, y, s, TOL[prec], "triangle64")


def test_method1_tt_ladder_full_size(ctx):
    A, B = W.tt_cores()
    spec = W.tt_ladder(A, B)
    p = tnsk.Params(m=1024, reps=64, seed=W.HASH_SEED)
    out, per = gpu_estimate(ctx, spec, p, torch.float32)
    y, s = oracle_estimate(spec, p, torch.float32)
    assert_parity(per, y, s, TOL[p.prec], "tt_ladder")


def test_method1_grid_bf16_inputs(ctx):
    spec = W.grid(3, 3, 4, seed=7)
    p = tnsk.Params(m=512, reps=8, seed=3)
    out, per = gpu_estimate(ctx, spec, p, torch.bfloat16)
    y, s = oracle_estimate(spec, p, torch.bfloat16)  # oracle on the bf16-rounded inputs
    assert_parity(per, y, s, TOL[p.prec], "grid bf16")


def test_method1_open_legs_many_shapes(ctx):
    rng = np.random.default_rng(21)
    for _ in range(6):
        spec = W.random_network(rng, p_range=(4, 7), dim_range=(2, 6), open_dim_range=(2, 5))
        p = tnsk.Params(m=128, reps=4, seed=int(rng.integers(1 << 30)))
        out, per = gpu_estimate(ctx, spec, p, torch.float32)
        y, s = oracle_estimate(spec, p, torch.float32)
        assert_parity(per, y, s, TOL[p.prec], "random open")


def _closed_specs():
    rng = np.random.default_rng(31)
    specs = [W.triangle(7, seed=2), W.grid(3, 3, 3, seed=5),
             W.NetSpec([rng.standard_normal((3, 2, 3)), rng.standard_normal(2)], [(0, 2), (1, 3)], [], "selftrace")]
    specs += [W.random_network(rng, p_range=(4, 9), dim_range=(2, 6), max_open=0) for _ in range(3)]
    return specs


@pytest.mark.parametrize("m", [64, 128, 256, 512, 1024])
def test_method1_warp_spectrum_every_size(ctx, m):
    """FP32 networks without open legs and 64 <= m <= 1024 take the warp-per-(network, rep)
    register FFT; every lane count per bin (J = m / 64) is covered."""
    for spec in _closed_specs():
        p = tnsk.Params(m=m, reps=5, seed=7 + m, prec=tnsk.PREC_FP32)
        out, per = gpu_estimate(ctx, spec, p, torch.float32)
        y, s = oracle_estimate(spec, p, torch.float32)
        assert_parity(per, y, s, TOL[p.prec], f"{spec.name} m={m}")


def test_method1_fiber_kernel(ctx):
    """FP32 tensors with a short last mode whose dim is not a multiple of 4 take the
    fiber kernel (whole fibers per thread): random networks of orders 2..7 with open
    legs (open last modes among them); an order-4 tensor with an open mode whose one
    item spans 19 batches of fibers (the FP32 accumulator between batches); the same
    network with its last mode on the complement side of the edge; a tensor of several
    chunks (items flushed by atomics); a 3000 x 7 tensor whose long mode's table is
    staged per chunk; an open last mode of dim 3; each against the oracle."""
    rng = np.random.default_rng(77)
    specs = [W.random_network(rng, p_range=(4, 8), dim_range=(2, 11), open_dim_range=(2, 5)) for _ in range(6)]
    big = rng.standard_normal((8, 40, 60, 9))
    A, Bm, v = rng.standard_normal((40, 5)), rng.standard_normal((60, 5)), rng.standard_normal(9)
    specs.append(W.NetSpec([big, A, Bm, v], [(1, 4), (2, 6), (5, 7), (3, 8)], [0], "fiber-multibatch"))
    specs.append(W.NetSpec([big, A, Bm, v], [(1, 4), (2, 6), (5, 7), (8, 3)], [0], "fiber-complement"))
    wide = rng.standard_normal((30, 20, 25, 9))
    specs.append(W.NetSpec([wide, rng.standard_normal((30, 20, 25)), rng.standard_normal(9)],
                           [(0, 4), (1, 5), (2, 6), (3, 7)], [], "fiber-chunks"))
    tall = rng.standard_normal((3000, 7))
    specs.append(W.NetSpec([tall, rng.standard_normal(3000), rng.standard_normal(7)], [(0, 2), (1, 3)], [],
                           "fiber-staged-ranges"))
    specs.append(W.NetSpec([rng.standard_normal((6, 5, 3)), rng.standard_normal((6, 5))], [(0, 3), (1, 4)], [2],
                           "fiber-open-last"))
    for i, spec in enumerate(specs):
        p = tnsk.Params(m=1024 if 6 <= i <= 8 else 256, reps=3, seed=70 + i)
        out, per = gpu_estimate(ctx, spec, p, torch.float32)
        y, sc = oracle_estimate(spec, p, torch.float32)
        assert_parity(per, y, sc, TOL[p.prec], f"{spec.name} m={p.m}")


@pytest.mark.parametrize("prec", [tnsk.PREC_FP32, tnsk.PREC_FP64])
def test_method1_mid_m_every_size(ctx, prec):
    """Closed networks at 2^11 <= m <= 2^14 (2^13 in FP64) take one CTA per sketch for the
    transforms and the product over blocks of the half spectra (more than one block of
    4096 bins from m = 2^13 on); every size against the oracle."""
    tdt = torch.float64 if prec == tnsk.PREC_FP64 else torch.float32
    top = 14 if prec == tnsk.PREC_FP32 else 13
    for l in range(11, top + 1):
        for spec in (W.grid(3, 3, 4, seed=11), _closed_specs()[3]):
            p = tnsk.Params(m=1 << l, reps=3, seed=90 + l, prec=prec)
            out, per = gpu_estimate(ctx, spec, p, tdt)
            y, s = oracle_estimate(spec, p, tdt)
            assert_parity(per, y, s, TOL[prec], f"{spec.name} m=2^{l}")


def test_method1_batch_mixes_spectrum_kernels(ctx):
    """One batch with networks for the warp kernel at two sizes, the per-sketch mid-m
    kernels (m = 2048, closed), the block kernel (open legs, m above 1024, m below 64), the
    large-m kernels and method 2, each against the oracle."""
    rng = np.random.default_rng(33)
    closed = _closed_specs()
    opened = [W.random_network(rng, p_range=(4, 6), dim_range=(2, 5), open_dim_range=(2, 4)) for _ in range(2)]
    specs = [closed[0], closed[1], opened[0], closed[3], opened[1], closed[4], closed[5], _trees()[2], closed[2],
             closed[0]]
    ms = [64, 1024, 256, 2048, 1024, 32, 256, 128, 1 << 15, 1 << 16]
    params = [tnsk.Params(m=m, reps=4 + (i % 3), seed=500 + i,
                          method=tnsk.ACYCLIC if s.name.startswith("tree") else tnsk.GENERAL)
              for i, (s, m) in enumerate(zip(specs, ms))]
    nets = [gpu_network(s, torch.float32) for s in specs]
    outs, pers, Os = [], [], []
    for s, p in zip(specs, params):
        dims = [d for x in s.tensors for d in np.shape(x)]
        O = int(np.prod([dims[g] for g in s.open])) if s.open else 1
        Os.append(O)
        outs.append(torch.zeros(max(O, 1), dtype=torch.float64, device="cuda"))
        pers.append(torch.zeros((p.reps, max(O, 1)), dtype=torch.float64, device="cuda"))
    ctx.estimate_batch(nets, params, outs, pers)
    ctx.sync()
    for s, p, pr, O in zip(specs, params, pers, Os):
        y, sc = oracle_estimate(s, p, torch.float32)
        assert_parity(pr.cpu().numpy()[:, :O], y, sc, TOL[p.prec], f"{s.name} m={p.m}")


@pytest.mark.parametrize("prec", [tnsk.PREC_FP32, tnsk.PREC_FP64])
@pytest.mark.parametrize("m", [1 << 14, 1 << 15, 1 << 16])
def test_method1_large_m(ctx, prec, m):
    """m above one CTA's shared memory (2^15, 2^16; 2^14 in FP64): two-pass FFT per sketch
    and the product over bin blocks, against the oracle."""
    tdt = torch.float64 if prec == tnsk.PREC_FP64 else torch.float32
    specs = [W.grid(3, 3, 4, seed=9), W.triangle(9, seed=3), _closed_specs()[3]]
    for spec in specs:
        p = tnsk.Params(m=m, reps=3, seed=77, prec=prec)
        out, per = gpu_estimate(ctx, spec, p, tdt)
        y, s = oracle_estimate(spec, p, tdt)
        assert_parity(per, y, s, TOL[prec], f"{spec.name} m={m}")


def test_large_m_limits(ctx):
    spec = _small_specs()[1]  # one open leg
    assert spec.open
    net = gpu_network(spec, torch.float32)
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(tnsk.TnskError) as e:  # open legs above the single-CTA FFT
        ctx.estimate(net, tnsk.Params(m=1 << 15, reps=2), out)
    assert e.value.status == -3
    with pytest.raises(tnsk.TnskError) as e:  # above 2^16
        ctx.estimate(gpu_network(W.triangle(4), torch.float32), tnsk.Params(m=1 << 17, reps=2), out)
    assert e.value.status == -3
    with pytest.raises(tnsk.TnskError) as e:  # method 2 stays within one CTA
        ctx.estimate(gpu_network(_trees()[1], torch.float32), tnsk.Params(m=1 << 15, reps=2, method=tnsk.ACYCLIC), out)
    assert e.value.status == -3


# ---------------------------------------------------------------- a5-a8 method 2
def _trees():
    rng = np.random.default_rng(5)
    specs = [W.random_tree(rng, p, dim_range=(2, 7), max_children=mc) for p, mc in
             [(2, 1), (3, 2), (6, 3), (9, 5), (12, 2)]]
    A, B = W.tt_cores(sites=5, bond=4, phys=3, seed=2)
    specs.append(W.tt_chain(A, B))
    return specs


@pytest.mark.parametrize("prec", [tnsk.PREC_FP32, tnsk.PREC_FP64])
@pytest.mark.parametrize("m", [1, 2, 32, 1024])
def test_method2_estimate_small(ctx, prec, m):
    tdt = torch.float64 if prec == tnsk.PREC_FP64 else torch.float32
    for spec in _trees():
        for root in (-1, 0, spec.p - 1):
            p = tnsk.Params(m=m, reps=5, seed=17, method=tnsk.ACYCLIC, root=root, prec=prec)
            out, per = gpu_estimate(ctx, spec, p, tdt)
            y, s = oracle_estimate(spec, p, tdt)
            assert_parity(per, y, s, TOL[prec], f"{spec.name} m={m} root={root}")


@pytest.mark.parametrize("root,reps,dtype", [(0, 70, "float32"), (3, 64, "float32"), (0, 16, "bfloat16")])
def test_method2_contraction_tile_edges(ctx, root, reps, dtype):
    """Row counts off the 128-row tile, columns off the 32-column chunk, reps off the
    64-rep tile, a parent mode that is not the first mode, BF16 inputs."""
    rng = np.random.default_rng(40 + root)
    X = [rng.standard_normal(300), rng.standard_normal((300, 200)), rng.standard_normal((170, 200)),
         rng.standard_normal(170)]
    spec = W.NetSpec(X, [(0, 1), (2, 4), (3, 5)], [], "chain-edges")
    tdt = getattr(torch, dtype)
    p = tnsk.Params(m=256, reps=reps, seed=9, method=tnsk.ACYCLIC, root=root)
    out, per = gpu_estimate(ctx, spec, p, tdt)
    y, s = oracle_estimate(spec, p, tdt)
    assert_parity(per, y, s, TOL[p.prec], f"chain-edges root={root} reps={reps} {dtype}")


def test_method2_tt_chain_full_size(ctx):
    A, B = W.tt_cores()
    spec = W.tt_chain(A, B)
    p = tnsk.Params(m=1024, reps=64, seed=W.HASH_SEED, method=tnsk.ACYCLIC)
    out, per = gpu_estimate(ctx, spec, p, torch.float32)
    y, s = oracle_estimate(spec, p, torch.float32)
    assert_parity(per, y, s, TOL[p.prec], "tt_chain")


def _rung_chain(sites, bond, phys, seed):
    """FP32 tensor-train cores, the oracle's dense chain of their rung merges (FP64 sums
    of the FP32 values), and the same chain for the library with the inner sites as
    grouped tensors (tnsk.Rung) and the two end vectors stored."""
    A, B = W.tt_cores(sites=sites, bond=bond, phys=phys, seed=seed)
    A = [a.astype(np.float32).astype(np.float64) for a in A]
    B = [b.astype(np.float32).astype(np.float64) for b in B]
    spec = W.tt_chain(A, B)
    ts = [torch.as_tensor(spec.tensors[0], dtype=torch.float32, device="cuda")]
    ts += [tnsk.Rung(torch.as_tensor(A[k], dtype=torch.float32, device="cuda"),
                     torch.as_tensor(B[k], dtype=torch.float32, device="cuda")) for k in range(1, sites - 1)]
    ts.append(torch.as_tensor(spec.tensors[-1], dtype=torch.float32, device="cuda"))
    return spec, tnsk.Network(ts, spec.edges, [])


@pytest.mark.parametrize("root", [0, -2])
def test_method2_grouped_rung_tensors(ctx, root):
    """Inner sites given as grouped tensors (entries formed inside the tensor-core sketch
    product, never stored) against the oracle on the dense merged chain, and against the
    library's own dense path; root 0 puts every parent mode first, the last site as root
    puts it second (the transposed form)."""
    sites = 5
    spec, net = _rung_chain(sites, 32, 8, seed=77)
    r = 0 if root == 0 else sites - 1
    p = tnsk.Params(m=1024, reps=16, seed=123, method=tnsk.ACYCLIC, root=r)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    per = torch.zeros((p.reps, 1), dtype=torch.float64, device="cuda")
    ctx.estimate(net, p, out, per)
    ctx.sync()
    y, sc = oracle_estimate(spec, p, torch.float32)
    assert_parity(per.cpu().numpy(), y, sc, TOL[p.prec], f"rung chain root={r}")
    _, per_dense = gpu_estimate(ctx, spec, p, torch.float32)
    assert np.all(np.abs(per.cpu().numpy() - per_dense) <= 1e-6 * sc)
    # a plan (CUDA-graph replays) gives the same estimates
    outp = torch.zeros(1, dtype=torch.float64, device="cuda")
    pl = ctx.plan([net], [p], [outp])
    for _ in range(3):
        pl.run()
    ctx.sync()
    assert abs(outp.item() - out.item()) <= 1e-6 * float(np.abs(sc).max())
    pl.close()


@pytest.mark.parametrize("root", [0, -2])
def test_grouped_rung_factored_tensor_cores_batch(ctx, root):
    """All factor dims 32 (the factored product on the tensor cores, one persistent CTA
    per SM): three chains with s = 8, 3 and 1 in one plan, 254 reps (a last block of 2
    reps), so that per height 192 blocks of 4 reps share 152 CTAs and CTAs cross from
    one node (and one s) to the next; both orientations, against the oracle on the
    dense merged chains, direct run and graph replays."""
    sites, R = 4, 254
    specs, nets = [], []
    for i, phys in enumerate((8, 3, 1)):
        spec, net = _rung_chain(sites, 32, phys, seed=300 + i)
        specs.append(spec)
        nets.append(net)
    r = 0 if root == 0 else sites - 1
    params = [tnsk.Params(m=256, reps=R, seed=40 + i, method=tnsk.ACYCLIC, root=r) for i in range(3)]
    outs = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in nets]
    pers = [torch.zeros((R, 1), dtype=torch.float64, device="cuda") for _ in nets]
    pl = ctx.plan(nets, params, outs, pers)
    want = [oracle_estimate(s, p, torch.float32) for s, p in zip(specs, params)]
    for run in range(3):
        pl.run()
        ctx.sync()
        for (y, sc), pr, s in zip(want, pers, specs):
            assert_parity(pr.cpu().numpy(), y, sc, TOL[tnsk.PREC_FP32], f"run {run} {s.name} root={r}")
    pl.close()


@pytest.mark.parametrize("root", [0, 2])
def test_grouped_rung_factored_small_dims(ctx, root):
    """Grouped tensor with factor dims below 32 and unequal (a, s, c) = (5, 3, 7),
    (b, s, d) = (6, 3, 4): the factored product (zero-padded tiles) against the oracle
    on the dense tensor; root 0 makes the row split (i, j), root 2 the transposed one."""
    rng = np.random.default_rng(91)
    A = rng.standard_normal((5, 3, 7)).astype(np.float32)
    B = rng.standard_normal((6, 3, 4)).astype(np.float32)
    X = np.einsum("isk,jsl->ijkl", A.astype(np.float64), B.astype(np.float64)).reshape(30, 28)
    x, y = rng.standard_normal(30), rng.standard_normal(28)
    spec = W.NetSpec([x, X, y], [(0, 1), (2, 3)], [], "rung-small")
    net = tnsk.Network([torch.as_tensor(x, dtype=torch.float32, device="cuda"),
                        tnsk.Rung(torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda")),
                        torch.as_tensor(y, dtype=torch.float32, device="cuda")], spec.edges, [])
    p = tnsk.Params(m=64, reps=11, seed=8, method=tnsk.ACYCLIC, root=root)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    per = torch.zeros((p.reps, 1), dtype=torch.float64, device="cuda")
    ctx.estimate(net, p, out, per)
    ctx.sync()
    y_o, sc = oracle_estimate(spec, p, torch.float32)
    assert_parity(per.cpu().numpy(), y_o, sc, TOL[p.prec], f"rung small root={root}")


@pytest.mark.parametrize("root", [0, -2])
def test_grouped_rung_factored_chain(ctx, root):
    """A chain of grouped tensors with bond 24 (below 32, not a multiple of 32: the
    factored product) against the oracle on the dense merged chain, both orientations."""
    sites = 5
    spec, net = _rung_chain(sites, 24, 4, seed=17)
    r = 0 if root == 0 else sites - 1
    p = tnsk.Params(m=512, reps=10, seed=33, method=tnsk.ACYCLIC, root=r)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    per = torch.zeros((p.reps, 1), dtype=torch.float64, device="cuda")
    ctx.estimate(net, p, out, per)
    ctx.sync()
    y, sc = oracle_estimate(spec, p, torch.float32)
    assert_parity(per.cpu().numpy(), y, sc, TOL[p.prec], f"rung chain bond 24 root={r}")


def test_grouped_rung_tensor_core_path(ctx):
    """Factor dims above 32 (bond 64, physical 2) take the tensor-core kernel that forms
    the entries: against the oracle on the dense merged chain."""
    spec, net = _rung_chain(4, 64, 2, seed=13)
    p = tnsk.Params(m=256, reps=8, seed=21, method=tnsk.ACYCLIC, root=0)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    per = torch.zeros((p.reps, 1), dtype=torch.float64, device="cuda")
    ctx.estimate(net, p, out, per)
    ctx.sync()
    y, sc = oracle_estimate(spec, p, torch.float32)
    assert_parity(per.cpu().numpy(), y, sc, TOL[p.prec], "rung chain bond 64")


def test_grouped_rung_tensors_rejected_where_unsupported(ctx):
    spec, net = _rung_chain(4, 32, 4, seed=5)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tnsk.TnskError):  # method 1 reads stored entries
        ctx.estimate(net, tnsk.Params(m=256, reps=4, method=tnsk.GENERAL), out)
    with pytest.raises(tnsk.TnskError):  # FP64 plans have no grouped-tensor product
        ctx.estimate(net, tnsk.Params(m=256, reps=4, method=tnsk.ACYCLIC, prec=tnsk.PREC_FP64), out)
    with pytest.raises(tnsk.TnskError):  # the grouped tensor as the root
        ctx.estimate(net, tnsk.Params(m=256, reps=4, method=tnsk.ACYCLIC, root=1), out)
    A, B = W.tt_cores(sites=4, bond=40, phys=4, seed=6)  # above 32 (tensor cores), 40: not a multiple of 32
    spec40 = W.tt_chain(A, B)
    ts = [torch.as_tensor(spec40.tensors[0], dtype=torch.float32, device="cuda")]
    ts += [tnsk.Rung(torch.as_tensor(A[k], dtype=torch.float32, device="cuda"),
                     torch.as_tensor(B[k], dtype=torch.float32, device="cuda")) for k in (1, 2)]
    ts.append(torch.as_tensor(spec40.tensors[-1], dtype=torch.float32, device="cuda"))
    with pytest.raises(tnsk.TnskError):
        ctx.estimate(tnsk.Network(ts, spec40.edges, []), tnsk.Params(m=256, reps=4, method=tnsk.ACYCLIC), out)


@pytest.mark.parametrize("prec", [tnsk.PREC_FP32, tnsk.PREC_FP64])
def test_entry_sharded_streams_sum_to_the_whole(ctx, prec):
    """The entries of a cyclic network with an open leg split between two streams (as
    two ranks would hold them): the streams' sketch buffers (tnsk_stream_sketches)
    match the oracle's sketches of each part, their sum estimates the whole, per rep,
    against the oracle on the full tensors."""
    rng = np.random.default_rng(52)
    X = [rng.standard_normal((6, 5)), rng.standard_normal((5, 7, 3)), rng.standard_normal((7, 6))]
    edges, open_ = [(1, 2), (3, 5), (6, 0)], [4]
    tdt = torch.float64 if prec == tnsk.PREC_FP64 else torch.float32
    spec = W.NetSpec(X, edges, open_, "entry-shards")
    Xr = rounded(spec, tdt)
    p = tnsk.Params(m=64, reps=6, seed=12, method=tnsk.GENERAL, prec=prec)
    bins, signs = oracle.m1_tables(Xr, edges, open_, seed=p.seed, reps=p.reps, m=p.m)
    streams, outs, pers = [], [], []
    for part in range(2):
        zeros = tnsk.Network([tnsk.Zeros(*x.shape, dtype=tdt) for x in Xr], edges, open_)
        out = torch.zeros(3, dtype=torch.float64, device="cuda")
        per = torch.zeros((p.reps, 3), dtype=torch.float64, device="cuda")
        st = ctx.stream(zeros, p, out, per)
        idx = [np.arange(x.size)[np.arange(x.size) % 2 == part] for x in Xr]
        tk = np.concatenate([np.full(i.size, k, np.int32) for k, i in enumerate(idx)])
        ti = np.concatenate(idx).astype(np.int64)
        dv = np.concatenate([x.reshape(-1)[i] for x, i in zip(Xr, idx)])
        st.update(torch.as_tensor(tk, device="cuda"), torch.as_tensor(ti, device="cuda"),
                  torch.as_tensor(dv, dtype=torch.float64, device="cuda"))
        ctx.sync()
        mine = [np.where(np.arange(x.size).reshape(x.shape) % 2 == part, x, 0.0) for x in Xr]
        want = oracle.m1_sketch(mine, edges, open_, p.m, bins, signs)
        scale = oracle.m1_sketch(Xr, edges, open_, p.m, bins, signs, abs_mode=True)
        got = st.sketches().double().cpu().numpy()[: want.size].reshape(want.shape)
        bound = sketch_tol(Xr, edges, open_, p.m, bins, signs, prec)
        assert np.all(np.abs(got - want) <= bound), f"part {part}"
        streams.append(st)
        outs.append(out)
        pers.append(per)
    xa, xb = streams[0].sketches(), streams[1].sketches()
    xa += xb  # the all-reduce of two ranks, on one GPU
    streams[0].estimate()
    ctx.sync()
    y, sc = oracle_estimate(spec, p, tdt)
    assert_parity(pers[0].cpu().numpy(), y, sc, TOL[prec], "entry-sharded sum")
    for st in streams:
        st.close()


@pytest.mark.parametrize("prec", [tnsk.PREC_FP32, tnsk.PREC_FP64])
def test_turnstile_stream_updates(ctx, prec):
    """Sec. 4.2's turnstile model: sketch a cyclic network with an open leg, apply
    batches of entry updates (repeated entries included) to the stored sketches, and
    re-estimate; each estimate against the oracle on the updated tensors."""
    rng = np.random.default_rng(31)
    X0 = [rng.standard_normal((6, 5)), rng.standard_normal((5, 7, 3)), rng.standard_normal((7, 6))]
    edges, open_ = [(1, 2), (3, 5), (6, 0)], [4]
    tdt = torch.float64 if prec == tnsk.PREC_FP64 else torch.float32
    spec0 = W.NetSpec(X0, edges, open_, "turnstile")
    p = tnsk.Params(m=64, reps=6, groups=2, seed=5, method=tnsk.GENERAL, prec=prec)
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    per = torch.zeros((p.reps, 3), dtype=torch.float64, device="cuda")
    st = ctx.stream(gpu_network(spec0, tdt), p, out, per)
    ctx.sync()
    y, sc = oracle_estimate(spec0, p, tdt)
    assert_parity(per.cpu().numpy(), y, sc, TOL[prec], "stream initial")
    X = [x.astype(np.float64) for x in rounded(spec0, tdt)]  # what the sketches hold
    for batch in range(2):
        n = 700
        k = rng.integers(0, 3, n)
        idx = np.array([rng.integers(0, X[kk].size) for kk in k])
        idx[: n // 10] = idx[n // 10: 2 * (n // 10)]  # repeated entries
        k[: n // 10] = k[n // 10: 2 * (n // 10)]
        delta = rng.standard_normal(n)
        for kk, ii, dd in zip(k, idx, delta):
            X[kk].reshape(-1)[ii] += dd
        st.update(torch.as_tensor(k, dtype=torch.int32, device="cuda"),
                  torch.as_tensor(idx, dtype=torch.int64, device="cuda"),
                  torch.as_tensor(delta, dtype=torch.float64, device="cuda"))
        st.estimate()
        ctx.sync()
        y, sc = oracle_estimate(W.NetSpec(X, edges, open_, "turnstile"), p, torch.float64)
        assert_parity(per.cpu().numpy(), y, sc, TOL[prec], f"stream after batch {batch}")
        assert np.allclose(out.cpu().numpy(), oracle.combine(per.cpu().numpy(), 2), rtol=1e-14, atol=0)
    # an update naming a tensor the network does not have is reported and changes nothing
    before = per.clone()
    st.update(torch.tensor([3], dtype=torch.int32, device="cuda"), torch.tensor([0], dtype=torch.int64, device="cuda"),
              torch.tensor([1.0], dtype=torch.float64, device="cuda"))
    with pytest.raises(tnsk.TnskError):
        ctx.sync()
    st.estimate()
    ctx.sync()
    assert torch.equal(per, before)
    st.close()
    with pytest.raises(tnsk.TnskError):  # method 2 keeps no per-tensor sketches
        ctx.stream(gpu_network(spec0, tdt), tnsk.Params(m=64, reps=2, method=tnsk.ACYCLIC), out)


def test_turnstile_sparse_triangle_count(ctx):
    """The sparse (COO) input path: tr(A^3) of a random graph's adjacency matrix from
    three all-zero tensors fed the nonzeros as updates, against the oracle's dense
    estimate with the same hashes."""
    rng = np.random.default_rng(33)
    n = 160
    Au = np.triu((rng.random((n, n)) < 0.15).astype(np.float64), 1)
    A = Au + Au.T
    spec = W.NetSpec([A, A, A], [(1, 2), (3, 4), (5, 0)], [], "triangles")
    p = tnsk.Params(m=256, reps=16, seed=9, method=tnsk.GENERAL)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    per = torch.zeros((p.reps, 1), dtype=torch.float64, device="cuda")
    st = ctx.stream(tnsk.Network([tnsk.Zeros(n, n)] * 3, spec.edges, []), p, out, per)
    rows, cols = np.nonzero(A)
    flat = (rows * n + cols).astype(np.int64)
    k = np.repeat(np.arange(3, dtype=np.int32), flat.size)
    st.update(torch.as_tensor(k, device="cuda"), torch.as_tensor(np.tile(flat, 3), device="cuda"),
              torch.ones(3 * flat.size, dtype=torch.float64, device="cuda"))
    st.estimate()
    ctx.sync()
    y, sc = oracle_estimate(spec, p, torch.float32)
    assert_parity(per.cpu().numpy(), y, sc, TOL[p.prec], "sparse triangles")
    assert np.allclose(out.cpu().numpy(), oracle.combine(per.cpu().numpy(), 1), rtol=1e-14, atol=0)
    st.close()


# ---------------------------------------------------------------- batch, combine, errors
def test_batch_matches_oracle_per_network(ctx):
    rng = np.random.default_rng(8)
    specs = [W.random_network(rng, p_range=(4, 6), dim_range=(2, 5), open_dim_range=(2, 4)) for _ in range(5)]
    specs += _trees()[:3]
    params = []
    for i, s in enumerate(specs):
        method = tnsk.ACYCLIC if s.name.startswith("tree") else tnsk.GENERAL
        params.append(tnsk.Params(m=64 << (i % 3), reps=4, groups=2, seed=1000 + i, method=method))
    nets = [gpu_network(s, torch.float32) for s in specs]
    outs, pers = [], []
    for s, p in zip(specs, params):
        dims = [d for x in s.tensors for d in np.shape(x)]
        O = int(np.prod([dims[g] for g in s.open])) if s.open else 1
        outs.append(torch.zeros(max(O, 1), dtype=torch.float64, device="cuda"))
        pers.append(torch.zeros((p.reps, max(O, 1)), dtype=torch.float64, device="cuda"))
    ctx.estimate_batch(nets, params, outs, pers)
    ctx.sync()
    for s, p, o, pr in zip(specs, params, outs, pers):
        y, sc = oracle_estimate(s, p, torch.float32)
        assert_parity(pr.cpu().numpy()[:, :y.shape[1]], y, sc, TOL[p.prec], s.name)
        assert np.allclose(o.cpu().numpy()[:y.shape[1]], oracle.combine(pr.cpu().numpy()[:, :y.shape[1]], 2),
                           rtol=1e-14, atol=0)


def test_uneven_random_networks_in_one_batch(ctx):
    """Networks of the uneven-batch family (4..12 tensors, degree 2..4, dims 2..16, 0..2
    open legs of dim 2..16, N(0,1)) in one planned batch, every per-rep entry against the
    oracle."""
    rng = np.random.default_rng(20260307)
    specs = [W.random_network(rng) for _ in range(40)]
    specs = [s for s in specs if sum(np.size(x) for x in s.tensors) < 2_000_000][:24]
    params = [tnsk.Params(m=256, reps=3, seed=0x7E57 + i) for i in range(len(specs))]
    nets = [gpu_network(s, torch.float32) for s in specs]
    Os = []
    for s in specs:
        dims = [d for x in s.tensors for d in np.shape(x)]
        Os.append(int(np.prod([dims[g] for g in s.open])) if s.open else 1)
    outs = [torch.zeros(max(O, 1), dtype=torch.float64, device="cuda") for O in Os]
    pers = [torch.zeros((3, max(O, 1)), dtype=torch.float64, device="cuda") for O in Os]
    plan = ctx.plan(nets, params, outs, pers)
    plan.run()
    ctx.sync()
    for s, p, pr, O in zip(specs, params, pers, Os):
        y, sc = oracle_estimate(s, p, torch.float32)
        assert_parity(pr.cpu().numpy()[:, :O], y, sc, TOL[p.prec], f"uneven {s.name}")
    plan.close()


def test_plan_runs_match_oracle_and_pick_up_new_data(ctx):
    rng = np.random.default_rng(12)
    specs = [W.random_network(rng, p_range=(4, 6), dim_range=(2, 5), open_dim_range=(2, 4)) for _ in range(3)]
    specs += _trees()[3:5]
    params = [tnsk.Params(m=128, reps=4, seed=50 + i,
                          method=tnsk.ACYCLIC if s.name.startswith("tree") else tnsk.GENERAL)
              for i, s in enumerate(specs)]
    nets = [gpu_network(s, torch.float32) for s in specs]
    Os = []
    for s in specs:
        dims = [d for x in s.tensors for d in np.shape(x)]
        Os.append(int(np.prod([dims[g] for g in s.open])) if s.open else 1)
    outs = [torch.zeros(max(O, 1), dtype=torch.float64, device="cuda") for O in Os]
    pers = [torch.zeros((p.reps, max(O, 1)), dtype=torch.float64, device="cuda") for p, O in zip(params, Os)]
    plan = ctx.plan(nets, params, outs, pers)
    for run in range(2):
        if run == 1:  # new values in the same buffers
            for s, n in zip(specs, nets):
                for k, t in enumerate(n.tensors):
                    s.tensors[k] = 2.0 * s.tensors[k]
                    t.copy_(torch.as_tensor(np.array(s.tensors[k], dtype=np.float64)).to(t.dtype))
        plan.run()
        ctx.sync()
        for s, p, pr, O in zip(specs, params, pers, Os):
            y, sc = oracle_estimate(s, p, torch.float32)
            assert_parity(pr.cpu().numpy()[:, :O], y, sc, TOL[p.prec], f"plan run {run} {s.name}")
    plan.close()


def test_plan_graph_replay_matches_direct_runs():
    """On a non-default stream a plan's runs from the second on replay one CUDA graph;
    every run matches the oracle and picks up new input values."""
    stream = torch.cuda.Stream()
    c = tnsk.Context(0, stream.cuda_stream)
    rng = np.random.default_rng(44)
    specs = [_closed_specs()[1], W.random_network(rng, p_range=(4, 6), dim_range=(2, 5), open_dim_range=(2, 3)),
             _trees()[3]]
    params = [tnsk.Params(m=m, reps=4, seed=90 + i, method=tnsk.ACYCLIC if s.name.startswith("tree") else tnsk.GENERAL)
              for i, (s, m) in enumerate(zip(specs, [256, 128, 64]))]
    with torch.cuda.stream(stream):
        nets = [gpu_network(s, torch.float32) for s in specs]
        Os = []
        for s in specs:
            dims = [d for x in s.tensors for d in np.shape(x)]
            Os.append(int(np.prod([dims[g] for g in s.open])) if s.open else 1)
        outs = [torch.zeros(max(O, 1), dtype=torch.float64, device="cuda") for O in Os]
        pers = [torch.zeros((p.reps, max(O, 1)), dtype=torch.float64, device="cuda") for p, O in zip(params, Os)]
    stream.synchronize()
    plan = c.plan(nets, params, outs, pers)
    for run in range(4):
        if run == 3:
            for s, n in zip(specs, nets):
                for k, t in enumerate(n.tensors):
                    s.tensors[k] = -1.5 * s.tensors[k]
                    t.copy_(torch.as_tensor(np.array(s.tensors[k], dtype=np.float64)).to(t.dtype))
            torch.cuda.synchronize()
        plan.run()
        c.sync()
        for s, p, pr, O in zip(specs, params, pers, Os):
            y, sc = oracle_estimate(s, p, torch.float32)
            assert_parity(pr.cpu().numpy()[:, :O], y, sc, TOL[p.prec], f"graph run {run} {s.name}")
    plan.close()
    c.close()


def test_rep0_blocks_match_the_whole_estimate(ctx):
    """tnsk_params.rep0: a call for reps [3, 7) gives reps 3..6 of the whole estimate."""
    for spec, method in [(_closed_specs()[1], tnsk.GENERAL), (_trees()[2], tnsk.ACYCLIC)]:
        whole = tnsk.Params(m=128, reps=8, seed=5, method=method)
        _, per_all = gpu_estimate(ctx, spec, whole, torch.float32)
        part = tnsk.Params(m=128, reps=4, seed=5, method=method, rep0=3)
        _, per_part = gpu_estimate(ctx, spec, part, torch.float32)
        y, sc = oracle_estimate(spec, whole, torch.float32)
        assert_parity(per_part, y[3:7], sc[3:7], TOL[tnsk.PREC_FP32], f"rep0 {spec.name}")
        assert_parity(per_all[3:7], y[3:7], sc[3:7], TOL[tnsk.PREC_FP32], f"whole {spec.name}")


@pytest.mark.parametrize("R,O,groups", [(12, 3, 4), (7, 1, 7), (64, 5, 1), (10, 2, 2)])
def test_combine_entry_point_matches_oracle(ctx, R, O, groups):
    rng = np.random.default_rng(R * 100 + O)
    per = rng.standard_normal((R, O))
    per_d = torch.as_tensor(per, device="cuda")
    out = torch.zeros(O, dtype=torch.float64, device="cuda")
    ctx.combine(per_d, groups, out)
    ctx.sync()
    assert np.array_equal(out.cpu().numpy(), oracle.combine(per, groups))


def test_estimate_sharded_on_one_rank_equals_estimate(ctx):
    from paper_2603_07387_gb300.sharding import estimate_sharded

    spec = _closed_specs()[0]
    p = tnsk.Params(m=64, reps=6, groups=3, seed=12)
    out, per = gpu_estimate(ctx, spec, p, torch.float32)
    net = gpu_network(spec, torch.float32)
    got = torch.zeros(1, dtype=torch.float64, device="cuda")
    allreps = estimate_sharded(ctx, net, p, got)
    ctx.sync()
    y, sc = oracle_estimate(spec, p, torch.float32)  # FP32 atomics: summation order varies run to run
    assert_parity(allreps.cpu().numpy(), y, sc, TOL[p.prec], "sharded")
    assert np.array_equal(got.cpu().numpy(), oracle.combine(allreps.cpu().numpy(), 3))


def test_degenerate_inputs(ctx):
    # scalars, an empty contracted mode, an empty open mode, a single self-contraction
    cases = [
        W.NetSpec([np.array(3.0), np.array(-2.0)], [], [], "scalars"),
        W.NetSpec([np.zeros((0, 3)), np.zeros((0,))], [(0, 2)], [1], "empty-contracted"),
        W.NetSpec([np.ones((2, 0)), np.ones(2)], [(0, 2)], [1], "empty-open"),
        W.NetSpec([np.arange(16.0).reshape(4, 4)], [(0, 1)], [], "trace"),
    ]
    for spec in cases:
        p = tnsk.Params(m=8, reps=3, seed=4)
        out, per = gpu_estimate(ctx, spec, p, torch.float32)
        y, s = oracle_estimate(spec, p, torch.float32)
        if y.size:
            assert_parity(per, y, s, TOL[p.prec], spec.name)
    p2 = tnsk.Params(m=8, reps=2, seed=4, method=tnsk.ACYCLIC)
    out, per = gpu_estimate(ctx, W.NetSpec([np.array(4.0)], [], [], "scalar"), p2, torch.float32)
    assert np.allclose(per, 4.0)


def test_errors_are_reported(ctx):
    A = [np.ones((3, 3)) for _ in range(3)]
    tri = W.NetSpec(A, [(1, 2), (3, 4), (5, 0)], [])
    net = gpu_network(tri, torch.float32)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(tnsk.TnskError) as e:
        ctx.estimate(net, tnsk.Params(m=8, reps=2, method=tnsk.ACYCLIC), out)
    assert e.value.status == -2
    with pytest.raises(tnsk.TnskError) as e:
        ctx.estimate(net, tnsk.Params(m=12, reps=2), out)
    assert e.value.status == -3
    with pytest.raises(tnsk.TnskError) as e:  # n_u != n_v
        xy = [torch.ones(3, device="cuda"), torch.ones(4, device="cuda")]
        ctx.estimate(tnsk.Network(xy, [(0, 1)], []), tnsk.Params(m=8, reps=2), out)
    assert e.value.status == -1
    with pytest.raises(tnsk.TnskError) as e:  # hyperedge (mode 1 in two contractions): not for method 2
        ctx.estimate(tnsk.Network(net.tensors, [(1, 2), (1, 4), (3, 5)], []),
                     tnsk.Params(m=8, reps=2, method=tnsk.ACYCLIC), out)
    assert e.value.status == -3
    with pytest.raises(tnsk.TnskError) as e:  # groups must divide reps
        ctx.estimate(net, tnsk.Params(m=8, reps=5, groups=2), out)
    assert e.value.status == -1
    ctx.sync()


# ---------------------------------------------------------------- exact pair contractions
def test_contract_pairs_match_the_exact_oracle(ctx):
    """tnsk_pairs: the tensor-train rung merge (M[a,b,c,d] = sum_s A[a,s,c] B[b,s,d]) at
    the bench's shapes, end sites, a pair sharing two modes, permuted outputs, FP64 /
    BF16 inputs (general path), a long last output mode."""
    rng = np.random.default_rng(61)
    cases = []
    cases.append((rng.standard_normal((32, 8, 32)), rng.standard_normal((32, 8, 32)), [1], [1], [0, 2, 1, 3],
                  torch.float32))
    cases.append((rng.standard_normal((6, 3, 5)), rng.standard_normal((4, 3, 7)), [1], [1], [0, 2, 1, 3],
                  torch.float32))
    cases.append((rng.standard_normal((3, 6)), rng.standard_normal((3, 4)), [0], [0], None, torch.float32))
    cases.append((rng.standard_normal((2, 5, 3)), rng.standard_normal((3, 2, 4)), [0, 2], [1, 0], [1, 0],
                  torch.float64))
    cases.append((rng.standard_normal((5, 4)), rng.standard_normal((6,)), [], [], [2, 0, 1], torch.bfloat16))
    cases.append((rng.standard_normal((3, 8, 4)), rng.standard_normal((8, 70)), [1], [0], None, torch.float32))
    # 20 rows sharing their B terms: a ragged group of the 16-byte-store path
    cases.append((rng.standard_normal((1, 4, 20)), rng.standard_normal((1, 4, 8)), [1], [1], [0, 2, 1, 3],
                  torch.float32))
    jobs, wants = [], []
    for A, B, am, bm, perm, dt in cases:
        Ad = torch.as_tensor(A).to(dt).cuda()
        Bd = torch.as_tensor(B).to(dt).cuda()
        Ar, Br = Ad.double().cpu().numpy(), Bd.double().cpu().numpy()
        na = Ar.ndim
        edges = [(a, na + b) for a, b in zip(am, bm)]
        free = [g for g in range(na) if g not in am] + [na + g for g in range(Br.ndim) if g not in bm]
        order = [free[i] for i in (perm if perm is not None else range(len(free)))]
        want = np.asarray(oracle.tc_einsum([Ar, Br], edges, order))
        out = torch.zeros(want.shape, dtype=torch.float32, device="cuda")
        jobs.append((Ad, Bd, am, bm, perm, out))
        terms = max(1, int(np.prod([Ar.shape[a] for a in am])))
        wants.append((want, float(np.abs(Ar).max() * np.abs(Br).max() * terms)))
    pr = ctx.pairs(jobs)
    for _ in range(2):  # a second run writes the same values
        pr.run()
        ctx.sync()
        for (A, B, am, bm, perm, out), (want, scale) in zip(jobs, wants):
            assert out.shape == want.shape
            assert np.allclose(out.cpu().numpy(), want, rtol=1e-5, atol=1e-6 * scale)
    pr.close()
    with pytest.raises(tnsk.TnskError):  # unequal shared dims
        ctx.contract_pairs([(jobs[1][0], jobs[1][1], [0], [0], None, jobs[1][5])])


def test_contract_pairs_many_jobs(ctx):
    """64 rung merges in one launch: fewer blocks per job than row groups, so every warp
    strides over several groups of 32 rows (an uneven number of them)."""
    rng = np.random.default_rng(62)
    jobs, wants = [], []
    for k in range(64):
        bond = 32 if k % 2 == 0 else 24
        A = rng.standard_normal((bond, 8, bond)).astype(np.float32)
        B = rng.standard_normal((bond, 8, bond)).astype(np.float32)
        want = np.einsum("asc,bsd->abcd", A.astype(np.float64), B.astype(np.float64))
        out = torch.zeros(want.shape, dtype=torch.float32, device="cuda")
        jobs.append((torch.as_tensor(A).cuda(), torch.as_tensor(B).cuda(), [1], [1], [0, 2, 1, 3], out))
        wants.append(want)
    pr = ctx.pairs(jobs)
    pr.run()
    ctx.sync()
    for (A, B, am, bm, perm, out), want in zip(jobs, wants):
        assert np.allclose(out.cpu().numpy(), want, rtol=1e-5, atol=1e-5 * 8 * np.abs(want).max())
    pr.close()


def test_plan_prelude_feeds_method2_beside_method1():
    """tnsk_plan_set_prelude: the rung merge attached to a plan runs ahead of method 2
    (the merged tensor is method 2's input) while method 1 sketches another network on
    the second stream; direct runs and graph replays match the oracle on the merged
    values, and new core values reach the estimate through the prelude."""
    stream = torch.cuda.Stream()
    c = tnsk.Context(0, stream.cuda_stream)
    rng = np.random.default_rng(47)
    A = rng.standard_normal((4, 3, 5))
    B = rng.standard_normal((6, 3, 7))
    vecs = [rng.standard_normal(n) for n in (4, 6, 5, 7)]
    m1_spec = W.random_network(rng, p_range=(4, 5), dim_range=(2, 5), open_dim_range=(2, 3))
    with torch.cuda.stream(stream):
        Ad = torch.as_tensor(A, dtype=torch.float32, device="cuda")
        Bd = torch.as_tensor(B, dtype=torch.float32, device="cuda")
        Md = torch.zeros((4, 6, 5, 7), dtype=torch.float32, device="cuda")
        vd = [torch.as_tensor(v, dtype=torch.float32, device="cuda") for v in vecs]
        # M[a, b, c, d] = sum_s A[a, s, c] B[b, s, d], contracted with one vector per mode
        star = tnsk.Network([Md] + vd, [(0, 4), (1, 5), (2, 6), (3, 7)], [])
        gen = gpu_network(m1_spec, torch.float32)
        dims = [d for x in m1_spec.tensors for d in np.shape(x)]
        O = int(np.prod([dims[g] for g in m1_spec.open])) if m1_spec.open else 1
        outs = [torch.zeros(1, dtype=torch.float64, device="cuda"), torch.zeros(max(O, 1), dtype=torch.float64,
                                                                               device="cuda")]
        pers = [torch.zeros((6, 1), dtype=torch.float64, device="cuda"),
                torch.zeros((6, max(O, 1)), dtype=torch.float64, device="cuda")]
    stream.synchronize()
    params = [tnsk.Params(m=64, reps=6, seed=31, method=tnsk.ACYCLIC),
              tnsk.Params(m=128, reps=6, seed=32, method=tnsk.GENERAL)]
    merge = c.pairs([(Ad, Bd, [1], [1], [0, 2, 1, 3], Md)])
    plan = c.plan([star, gen], params, outs, pers)
    plan.set_prelude(merge)
    for run in range(4):
        if run == 2:  # new core values: only the prelude carries them into M
            A = -0.5 * A
            with torch.cuda.stream(stream):
                Ad.copy_(torch.as_tensor(A, dtype=torch.float32, device="cuda"))
        plan.run()
        c.sync()
        M = Md.double().cpu().numpy()
        want = np.einsum("asc,bsd->abcd", np.float32(A).astype(np.float64), np.float32(B).astype(np.float64))
        assert np.allclose(M, want, rtol=1e-5, atol=1e-6 * np.abs(want).max()), f"run {run}: merged tensor"
        star_spec = W.NetSpec([M] + [np.float32(v).astype(np.float64) for v in vecs],
                              [(0, 4), (1, 5), (2, 6), (3, 7)], [], "star")
        y, sc = oracle_estimate(star_spec, params[0], torch.float64)
        assert_parity(pers[0].cpu().numpy(), y, sc, TOL[tnsk.PREC_FP32], f"prelude run {run}: method 2")
        y, sc = oracle_estimate(m1_spec, params[1], torch.float32)
        assert_parity(pers[1].cpu().numpy()[:, :O], y, sc, TOL[tnsk.PREC_FP32], f"prelude run {run}: method 1")
    plan.set_prelude(None)  # detached: M keeps its last values
    A2 = 3.0 * A
    with torch.cuda.stream(stream):
        Ad.copy_(torch.as_tensor(A2, dtype=torch.float32, device="cuda"))
    plan.run()
    c.sync()
    assert np.allclose(Md.double().cpu().numpy(), M)
    plan.close()
    merge.close()
    c.close()
