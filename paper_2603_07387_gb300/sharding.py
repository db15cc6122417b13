"""One estimate's repetitions over several ranks (one process per GPU).

Repetitions are independent: rep r draws its hash functions from (seed, r) alone
(tnsk_params.rep0 offsets the block a call draws). So rank k of W estimates the
contiguous block of reps ``rep_shard(R, W, k)``, and the one exchange of the path
is a gather of those per-rep FP64 estimates, in rep order, onto every rank; the
median of group means (Theorem 1) then runs on the gathered array exactly as in a
single-GPU call (``Context.combine``), so the sharded result equals the unsharded
one. Batches of independent networks need no exchange at all: each rank takes
its own networks.

A tensor too large for one GPU is split by entries instead: sketches are linear in
the tensors (Sec. 4.2), so ranks that sketch disjoint parts of the same tensors'
entries (turnstile streams with the same network and params) hold sketches that sum
to those of the whole; one all-reduce of the sketch buffers (reps x sum_k O_k m
values) precedes the transform, product and combination (``allreduce_sketches``).
"""
from __future__ import annotations

import dataclasses


def rep_shard(reps: int, world: int, rank: int) -> tuple[int, int]:
    """Rank ``rank``'s contiguous block [r0, r1) of ``reps`` repetitions; blocks are in
    rank order, cover every rep once, and differ in size by at most one."""
    if reps < 0 or world < 1 or not 0 <= rank < world:
        raise ValueError("need reps >= 0, world >= 1, 0 <= rank < world")
    q, extra = divmod(reps, world)
    r0 = rank * q + min(rank, extra)
    return r0, r0 + q + (1 if rank < extra else 0)


def gather_reps(local, reps: int, group=None):
    """All ranks' per-rep blocks [r1 - r0][O] (torch FP64, on the collective's
    device) gathered in rep order into [reps][O] on every rank."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    if world == 1:
        return local.contiguous()
    O = local.shape[1]
    width = -(-reps // world)  # the largest block
    pad = torch.zeros((width, O), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    blocks = []
    for k in range(world):
        r0, r1 = rep_shard(reps, world, k)
        blocks.append(parts[k][: r1 - r0])
    return torch.cat(blocks, dim=0).contiguous()


def allreduce_sketches(x, group=None):
    """Sums the sketch buffer ``x`` (a torch tensor: ``Stream.sketches()`` on the GPU,
    or any tensor the collective's backend takes) over the ranks of ``group`` in place.
    On the GPU the stream's work must be ordered before it: the library's ctx runs on
    torch's current stream, or the caller synchronises first."""
    import torch.distributed as dist

    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(x, op=dist.ReduceOp.SUM, group=group)
    return x


def estimate_entry_sharded(stream, group=None):
    """The estimate of the whole from this rank's turnstile stream over its part of the
    entries: all-reduce of the sketches, then ``stream.estimate()`` (outputs as the
    stream was created with, the same on every rank)."""
    allreduce_sketches(stream.sketches(), group)
    stream.estimate()


def estimate_sharded(ctx, net, params, out, group=None):
    """tnsk_estimate of one network with its reps split over the ranks of ``group``:
    each rank runs its block of reps (``rep0`` offset), the per-rep estimates are
    gathered, and ``ctx.combine`` takes the median of group means into ``out``
    (device FP64, the network's output entries) on every rank."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    r0, r1 = rep_shard(params.reps, world, rank)
    O = out.numel()
    local = torch.zeros((r1 - r0, O), dtype=torch.float64, device=out.device)
    if r1 > r0:
        shard = dataclasses.replace(params, reps=r1 - r0, rep0=params.rep0 + r0, groups=1)
        scratch = torch.zeros(O, dtype=torch.float64, device=out.device)
        ctx.estimate(net, shard, scratch, local)
    allreps = gather_reps(local, params.reps, group)
    ctx.combine(allreps, params.groups, out)
    return allreps
