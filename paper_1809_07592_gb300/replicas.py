"""Multi-GPU deployment by replicas: blocks are independent, so each rank (one
process per GPU) hashes its own share with no collective on the data path. The
only cross-rank step is the timing reduction (max over ranks) of a benchmark.
"""
from __future__ import annotations


def shard(count: int, rank: int, world: int) -> range:
    """Contiguous share of `count` independent items for `rank` of `world` (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(count, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def rank_base_seed(rank: int, stride: int = 1000) -> int:
    """Input-generator base seed of a rank, so replicas hash distinct synthetic keys."""
    return stride * rank


def max_over_ranks(value: float, device=None) -> float:
    """All-reduce MAX of a scalar over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Aggregate throughput: units every rank processed / the slowest rank's time."""
    return units_per_rank * world / max_seconds
