"""Repetitions of one estimate split over ranks: the shard arithmetic, and the
exchange (a gather of per-rep estimates in rep order) run as two gloo ranks on the
CPU; the per-rep values come from the oracle, drawn for each rank's block of reps."""
import os

import numpy as np
import pytest

from paper_2603_07387_gb300.sharding import gather_reps, rep_shard


@pytest.mark.parametrize("reps,world", [(64, 2), (7, 2), (5, 4), (1, 3), (0, 2), (65536, 8)])
def test_rep_shard_covers_every_rep_once_in_order(reps, world):
    blocks = [rep_shard(reps, world, k) for k in range(world)]
    assert blocks[0][0] == 0 and blocks[-1][1] == reps
    for (a0, a1), (b0, b1) in zip(blocks, blocks[1:]):
        assert a1 == b0
    sizes = [b - a for a, b in blocks]
    assert max(sizes) - min(sizes) <= 1 and all(s >= 0 for s in sizes)


def test_rep_shard_rejects_bad_arguments():
    for args in [(-1, 2, 0), (4, 0, 0), (4, 2, 2), (4, 2, -1)]:
        with pytest.raises(ValueError):
            rep_shard(*args)


def _rank_main(rank, world, port, reps, groups, result_path):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2603_07387_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec = W.triangle(6, seed=4)
        r0, r1 = rep_shard(reps, world, rank)
        # this rank's block of reps: reps r0 .. r1 - 1 of the same seed
        y, _ = oracle.m1_estimate(spec.tensors, spec.edges, spec.open, m=16, reps=r1, seed=31)
        local = torch.as_tensor(y[r0:r1], dtype=torch.float64)
        allreps = gather_reps(local, reps).numpy()
        np.save(f"{result_path}.{rank}.npy", allreps)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("reps,groups", [(12, 3), (7, 7), (9, 1)])
def test_two_gloo_ranks_gather_reps_and_combine_like_one(tmp_path, reps, groups):
    import socket

    import torch.multiprocessing as mp

    import oracle
    from paper_2603_07387_gb300 import workloads as W

    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        port = sck.getsockname()[1]
    world = 2
    path = str(tmp_path / "gathered")
    mp.start_processes(_rank_main, args=(world, port, reps, groups, path), nprocs=world, join=True,
                       start_method="spawn")
    spec = W.triangle(6, seed=4)
    y_all, _ = oracle.m1_estimate(spec.tensors, spec.edges, spec.open, m=16, reps=reps, seed=31)
    for rank in range(world):
        got = np.load(f"{path}.{rank}.npy")
        assert got.shape == y_all.shape
        assert np.array_equal(got, y_all)  # same reps, same order, bit for bit
        assert np.array_equal(oracle.combine(got, groups), oracle.combine(y_all, groups))


def _sketch_rank_main(rank, world, port, result_path):
    """Rank k sketches its half of the entries of a triangle network with an open leg
    (the other entries zero) with the oracle, and the ranks all-reduce the sketches."""
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2603_07387_gb300 import workloads as W
    from paper_2603_07387_gb300.sharding import allreduce_sketches

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, edges, open_ = _entry_split_net()
        mine = [np.where(np.arange(x.size).reshape(x.shape) % world == rank, x, 0.0) for x in X]
        bins, signs = oracle.m1_tables(X, edges, open_, seed=9, reps=5, m=32)
        x = torch.as_tensor(oracle.m1_sketch(mine, edges, open_, 32, bins, signs))
        allreduce_sketches(x)
        np.save(f"{result_path}.{rank}.npy", x.numpy())
    finally:
        dist.destroy_process_group()


def _entry_split_net():
    rng = np.random.default_rng(8)
    X = [rng.standard_normal((5, 4)), rng.standard_normal((4, 3, 6)), rng.standard_normal((6, 5))]
    return X, [(1, 2), (4, 5), (6, 0)], [3]


def test_two_gloo_ranks_sum_entry_shard_sketches(tmp_path):
    """Entries split over two ranks: the all-reduced sketches equal the sketches of the
    whole tensors (linearity), and the estimate from them (the paper's e_1^T F^-1 of
    the Hadamard product, per open entry) equals the oracle's estimate of the whole."""
    import socket

    import torch.multiprocessing as mp

    import oracle

    with socket.socket() as sck:
        sck.bind(("127.0.0.1", 0))
        port = sck.getsockname()[1]
    world = 2
    path = str(tmp_path / "sk")
    mp.start_processes(_sketch_rank_main, args=(world, port, path), nprocs=world, join=True, start_method="spawn")
    X, edges, open_ = _entry_split_net()
    m, R = 32, 5
    bins, signs = oracle.m1_tables(X, edges, open_, seed=9, reps=R, m=m)
    whole = oracle.m1_sketch(X, edges, open_, m, bins, signs)
    for rank in range(world):
        got = np.load(f"{path}.{rank}.npy")
        assert np.allclose(got, whole, rtol=1e-12, atol=1e-12)
    # estimate from the summed sketches: tensor 1 holds the open leg (O_1 = 3 sketches)
    got = np.load(f"{path}.0.npy").reshape(R, -1)
    y_ref, _ = oracle.m1_estimate(X, edges, open_, m=m, reps=R, seed=9)
    for r in range(R):
        x0, x1, x2 = got[r, :m], got[r, m:4 * m].reshape(3, m), got[r, 4 * m:5 * m]
        F = np.fft.fft
        y = [np.real(np.sum(F(x0) * F(x1[o]) * F(x2))) / m for o in range(3)]
        assert np.allclose(y, y_ref[r], rtol=1e-10, atol=1e-10)
