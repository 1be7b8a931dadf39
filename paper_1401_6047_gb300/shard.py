"""Work split over ranks for the multi-GPU sweep and surrogate runs.

Parameter points are independent, so N ranks split them with no exchange
on the data path: rank r takes every N-th point of the cost-sorted list
(points of similar cost spread evenly), runs them on its own GPU, and the
only collectives are a barrier around the timed region and the maximum of
the ranks' times (plus, when results are wanted on one rank, a gather).
"""
from __future__ import annotations

from typing import Sequence


def split(n: int, rank: int, world: int, cost: Sequence[float] | None = None) -> list[int]:
    """Indices of the points rank `rank` of `world` runs: sorted by cost
    (descending, ties by index) when costs are given, then dealt round-robin
    so every rank gets a similar mix."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in 0..world-1")
    order = list(range(n))
    if cost is not None:
        if len(cost) != n:
            raise ValueError("one cost per point")
        order.sort(key=lambda i: (-float(cost[i]), i))
    return order[rank::world]


def slowest(seconds: float, group=None) -> float:
    """The largest of the ranks' times (all_reduce MAX); the value itself
    when no process group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(seconds)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
