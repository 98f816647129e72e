"""Replica-parallel host logic: images are independent, so N GPUs run N
replicas of the same path on disjoint shares of the images, with no data-path
collective.  torch.distributed is used only to agree on timing (a barrier and
a max over ranks), with NCCL on GPUs or gloo on the host.
"""

from __future__ import annotations

from typing import Sequence


def shard(items: Sequence, rank: int, world: int) -> list:
    """Round-robin share of `items` for `rank` of `world` (every item exactly once)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of world {world}")
    return list(items[rank::world])


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the slowest replica sets the time).
    Without an initialised process group this is the value itself."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, seconds_max: float, world: int) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    if seconds_max <= 0:
        raise ValueError("time must be positive")
    return units_per_rank * world / seconds_max
