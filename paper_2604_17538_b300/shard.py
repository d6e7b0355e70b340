"""Data-parallel sharding of the contact path over ranks (one process per GPU).

Body pairs are independent and every reduction of the method (a group's blend,
a pair's gradient) stays inside one pair, so ranks share nothing on the data
path: each rank generates and runs its own shard of environments from its own
seed stream, and the only collectives are a barrier around the timed region
and the reductions of the timing (max over ranks) and of the work done (sum
over ranks) that turn per-rank measurements into one whole-job rate.

A caller that splits one global list of pairs over the ranks instead takes a
contiguous range of pairs per rank (``shard_range``) and, after the step,
gathers the ranks' output rows on one rank in global pair order
(``gather_rows``): the host-side gather is the only exchange.
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


def shard_range(n_pairs: int, rank: int, world: int):
    """Contiguous pairs [lo, hi) of rank `rank` when n_pairs are split over
    `world` ranks: the first n_pairs % world ranks take one pair more."""
    q, r = divmod(int(n_pairs), int(world))
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def gather_rows(local, dst: int = 0):
    """Concatenates every rank's row block (a numpy array, rows = its pairs'
    outputs in pair order) on rank `dst`, in rank order -- the global pair
    order of ``shard_range``.  Returns the array on `dst`, None elsewhere (the
    block itself on one rank)."""
    import numpy as np
    d = _dist()
    if d is None or d.get_world_size() == 1:
        return local
    blocks = [None] * d.get_world_size() if d.get_rank() == dst else None
    d.gather_object(local, blocks, dst=dst)
    if d.get_rank() != dst:
        return None
    return np.concatenate(blocks, axis=0)
