"""Multi-GPU layout of the decode benchmarks: independent replicas, one process per GPU.

Scenes are independent (and so are the lanes inside a scene), so the decode needs no data
exchange between GPUs: each rank decodes its own scenes, and the only collective is the
timing reduction (the slowest rank sets the job's time).  Ranks, world size and the local
GPU come from the torchrun environment.
"""
from __future__ import annotations

import os


def rank_info() -> tuple[int, int, int]:
    """(rank, world size, local rank) from RANK / WORLD_SIZE / LOCAL_RANK (default 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n: int, rank: int, world: int) -> range:
    """The items of rank `rank` when n independent items are split as evenly as possible:
    rank r takes [floor(r n / world), floor((r + 1) n / world))."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    return range(rank * n // world, (rank + 1) * n // world)


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of `value` over all ranks (the value itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """The sum of `value` over all ranks (units decoded by the whole job)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
