"""Host logic of the multi-GPU mode: replicas with no data exchange.

Video streams are independent (each carries its own chaining state), so N
GPUs serve N disjoint sets of streams; nothing of the cipher crosses GPUs.
Ranks only agree on the timing of a measured region: a barrier before and
after it, and the maximum elapsed time over ranks, which is what a job-level
throughput must divide by.  Works with any torch.distributed backend (NCCL on
GPUs, gloo on CPU for the tests)."""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_streams(n_streams: int, rank: int, world: int) -> list[int]:
    """Stream ids owned by `rank`: a balanced contiguous block."""
    lo = (n_streams * rank) // world
    hi = (n_streams * (rank + 1)) // world
    return list(range(lo, hi))


def max_over_ranks(value_ms: float, device=None) -> float:
    """Maximum of a per-rank elapsed time (ms) over all ranks (identity when not distributed)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value_ms)
    t = torch.tensor([float(value_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: list[int] | int, max_ms: float, world: int = 1) -> float:
    """Units per second of the whole job: all ranks' units over the slowest rank's time."""
    units = sum(units_per_rank) if isinstance(units_per_rank, list) else units_per_rank * world
    return units / (max_ms / 1000.0)
