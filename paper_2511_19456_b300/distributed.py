"""Multi-GPU use: points are independent, so a job shards its points across
ranks (one process per GPU) and needs no collective on the data path.  The
only collectives are host-side bookkeeping: the timing maximum over ranks and,
for Monte Carlo integration, the sum of per-rank partial sums.
"""
from __future__ import annotations


def shard(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous [start, stop) share of n_total points for `rank` of `world`;
    shares differ by at most one point."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def _reduce(value: float, op: str, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(value: float, device=None) -> float:
    return _reduce(value, "max", device)


def sum_over_ranks(value: float, device=None) -> float:
    return _reduce(value, "sum", device)


def mc_mean(local_sum: float, local_count: int, device=None) -> float:
    """Global mean of a Monte Carlo estimate from per-rank partial sums."""
    return sum_over_ranks(local_sum, device) / sum_over_ranks(float(local_count), device)
