"""Multi-GPU plumbing for independent replicas.

The strict SGD_Tucker step (Algorithm 1) is a chain of dependent phases per
minibatch, so one decomposition is not split across GPUs; N GPUs run N
independent problems (replicas of a workload, or disjoint sets of tensors of
a batched workload) with no data-path collective.  torch.distributed is only
used for the start/stop barrier and the max-over-ranks timing.
"""
from __future__ import annotations

import os
from typing import List, Sequence, Tuple


def world() -> Tuple[int, int, int]:
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str) -> None:
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend)


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of `value` over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def weak_scaling_rate(units_per_rank: float, seconds_per_rank: float, device=None) -> Tuple[float, float]:
    """Whole-job throughput: all ranks' units over the slowest rank's time.
    Returns (rate, max_seconds)."""
    total = sum_over_ranks(units_per_rank, device)
    tmax = max_over_ranks(seconds_per_rank, device)
    return (total / tmax if tmax > 0 else 0.0), tmax


def shard(weights: Sequence[float], world_size: int, rank: int) -> List[int]:
    """Indices of the items assigned to `rank`: greedy longest-processing-time
    assignment by weight (ties by index), identical on every rank."""
    order = sorted(range(len(weights)), key=lambda i: (-float(weights[i]), i))
    load = [0.0] * world_size
    owner = [0] * len(weights)
    for i in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += float(weights[i])
    return [i for i in range(len(weights)) if owner[i] == rank]
