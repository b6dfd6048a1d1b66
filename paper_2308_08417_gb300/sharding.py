"""Splitting a batch across GPUs (one process per GPU).

Systems are independent, and the paper notes that distributing them over
ranks needs no communication (Sec. 5.2): rank r solves a contiguous range of
systems and nothing is exchanged on the data path. The only collective a run
needs is host-side bookkeeping, such as the slowest rank's time.
"""

from __future__ import annotations


def shard_range(num_batch: int, rank: int, world: int) -> tuple[int, int]:
    """[begin, end) of the systems rank `rank` of `world` solves: contiguous,
    sizes differing by at most one, covering every system exactly once."""
    if world < 1 or not 0 <= rank < world or num_batch < 0:
        raise ValueError("need 0 <= rank < world and num_batch >= 0")
    base, extra = divmod(num_batch, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def cost_shard_range(costs, rank: int, world: int) -> tuple[int, int]:
    """[begin, end) of a contiguous split of systems with per-system cost
    estimates `costs` (uneven batches): boundary r is the first system whose
    cumulative cost reaches r / world of the total, so every rank gets about
    the same work. Covers every system exactly once; with equal costs it
    matches shard_range up to rounding."""
    import numpy as np

    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    c = np.asarray(costs, dtype=np.float64)
    if c.ndim != 1 or (c < 0).any():
        raise ValueError("costs must be a 1-D array of non-negative numbers")
    total = np.concatenate([[0.0], np.cumsum(c)])

    def cut(r):
        if r <= 0:
            return 0
        if r >= world:
            return len(c)
        return int(np.searchsorted(total, total[-1] * r / world, side="left"))

    return cut(rank), cut(rank + 1)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
