"""Data-parallel sharding of the contact path over ranks (one process per GPU).

Body pairs are independent and every reduction of the method (a group's blend,
a pair's gradient) stays inside one pair, so ranks share nothing on the data
path: each rank generates and runs its own shard of environments from its own
seed stream, and the only collectives are a barrier around the timed region
and the reductions of the timing (max over ranks) and of the work done (sum
over ranks) that turn per-rank measurements into one whole-job rate.
"""
from __future__ import annotations


def shard_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s shard (disjoint seed streams per rank)."""
    return int(base) + 1000 * int(rank)


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def reduce_max(values, device="cpu"):
    """Element-wise max over ranks of a list of floats (identity on one rank)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    d = _dist()
    if d is not None and d.get_world_size() > 1:
        d.all_reduce(t, op=d.ReduceOp.MAX)
    return t.tolist()


def reduce_sum(values, device="cpu"):
    """Element-wise sum over ranks of a list of numbers (identity on one rank)."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    d = _dist()
    if d is not None and d.get_world_size() > 1:
        d.all_reduce(t, op=d.ReduceOp.SUM)
    return t.tolist()


def job_rate(units_local, seconds_local, device="cpu"):
    """(total units, slowest rank's seconds, total units / slowest seconds):
    the whole-job throughput of ranks that each processed `units_local` in
    `seconds_local`."""
    (units,) = reduce_sum([units_local], device)
    (secs,) = reduce_max([seconds_local], device)
    return units, secs, units / secs
