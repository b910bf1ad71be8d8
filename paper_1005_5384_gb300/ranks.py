"""Host-side logic of a multi-GPU run (one process per GPU, torch.distributed).

The force calculation shards by independent problems: every rank computes its
own systems and no data-path collective exists. What the ranks share is
bookkeeping: which systems a rank owns, and the whole-job rate, taken over
the slowest rank. These helpers are backend-agnostic (NCCL on GPUs, gloo on
CPUs for the tests).
"""
from __future__ import annotations

import numpy as np


def rank_seed(seed: int, rank: int) -> int:
    """Seed of the independent system a rank generates (replica runs)."""
    return int(seed) + int(rank)


def shard_systems(sizes, rank: int, world: int):
    """Contiguous range [lo, hi) of system indices owned by `rank`, chosen so
    that the ranks' particle counts are as equal as the order allows: rank r
    takes the systems whose cumulative count midpoints fall in the r-th of
    `world` equal slices of the total."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    if sizes.size == 0:
        return 0, 0
    cum = np.concatenate([[0], np.cumsum(sizes)])
    mid = 0.5 * (cum[:-1] + cum[1:])
    owner = np.minimum((mid * world // cum[-1]).astype(np.int64), world - 1)
    idx = np.nonzero(owner == rank)[0]
    if idx.size == 0:
        lo = int(np.searchsorted(owner, rank))
        return lo, lo
    return int(idx[0]), int(idx[-1]) + 1


def max_over_ranks(dist, value: float, device=None) -> float:
    """Maximum of `value` over all ranks (the slowest rank's time); the value
    itself when `dist` is None."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value: float, device=None) -> float:
    """Sum of `value` over all ranks (units processed by the whole job)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(dist, units: float, seconds: float, device=None) -> float:
    """Whole-job throughput: units processed by all ranks / the slowest rank's time."""
    return sum_over_ranks(dist, units, device) / max_over_ranks(dist, seconds, device)
