"""Multi-GPU replicas: independent fields sharded across ranks.

The extremum graph of one field never needs data from another field, so a
batch shards by field with no collective on the data path: each rank (one
process per GPU) computes the fields assigned to it.  The only communication
is for reporting: the maximum step time over ranks (the job's wall time) and
sums of processed vertices.  One large field would instead shard as slabs
along the slowest axis with a one-layer halo exchange; that path is not
built (every box in use has a single GPU).
"""
from __future__ import annotations

from typing import List, Sequence


def shard(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Deterministic longest-processing-time assignment of items (by vertex
    count) to `world` ranks; returns the item indices of every rank, each
    list in ascending index order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += int(sizes[i])
    return [sorted(x) for x in out]


def my_share(sizes: Sequence[int], rank: int, world: int) -> List[int]:
    return shard(sizes, world)[rank]


def _dist():
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            return dist
    except Exception:
        pass
    return None


def reduce_max(value: float, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (identity without a group)."""
    dist = _dist()
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, device=None) -> float:
    dist = _dist()
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
