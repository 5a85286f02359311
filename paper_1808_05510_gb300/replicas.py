"""Whole-job numbers when one process per GPU runs its own share of the work.

A single greedy solve does not shard (each rank step depends on the previous
residual, each PCG iteration on a global inner product), so several GPUs run
independent replicas, or independent members of a lambda x fold sweep.  The
only exchanges are host-side: the scalars that make the whole-job number
(work summed over ranks, time of the slowest rank) and the per-member scores
of a sweep.  Nothing here touches the solver's data.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def aggregate(units_local: float, ms_local: float, world: int, device="cpu") -> Tuple[float, float]:
    """(units summed over ranks, milliseconds of the slowest rank).  With world
    > 1 the process group must be initialised (gloo with device "cpu", nccl
    with a CUDA device)."""
    import torch

    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist

        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def shard_members(members: Sequence, rank: int, world: int) -> List:
    """The members rank `rank` of `world` solves: every world-th member in
    longest-first order (largest lambda first), so that every rank gets the same
    mix of costly and cheap members.  The shards are disjoint and cover all."""
    order = sorted(range(len(members)), key=lambda k: -members[k][0])
    return [members[k] for k in order[rank::world]]


def gather_objects(obj, world: int) -> list:
    """Every rank's `obj`, in rank order (the rank's own when world == 1)."""
    if world <= 1:
        return [obj]
    import torch.distributed as dist

    out = [None] * world
    dist.all_gather_object(out, obj)
    return out
