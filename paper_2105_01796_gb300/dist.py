"""Host-side multi-GPU logic: one process per GPU, tracks sharded across ranks.

Tracks are independent (paper Sect. 4.1: track-level parallelism; Sect. 6: a
team of host threads, one GPU each), so a batch splits into contiguous track
ranges with no exchange on the data path.  The only collectives are a
maximum over ranks for timing and, for alignment gradients, one sum of the
per-surface gradient vector.  Works with the NCCL backend (GPU tensors) and
the gloo backend (CPU tensors).
"""
from __future__ import annotations

import numpy as np


def shard_range(n_tracks: int, rank: int, world: int, offsets=None):
    """[begin, end) of the tracks of `rank`.

    Without offsets the ranges have equal track counts (±1).  With offsets
    (int array of n_tracks + 1) the cut points balance the number of states
    (the work) per rank instead."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    if offsets is None:
        b = n_tracks * rank // world
        e = n_tracks * (rank + 1) // world
        return int(b), int(e)
    o = np.asarray(offsets, dtype=np.int64)
    total = int(o[-1] - o[0])

    def cut(r):
        if r == 0:
            return 0
        if r == world:
            return n_tracks
        target = o[0] + total * r // world
        return int(np.searchsorted(o[:-1], target, side="left"))

    return cut(rank), cut(rank + 1)


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(grad):
    """In-place sum of a gradient tensor over all ranks (one all-reduce)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(grad, op=dist.ReduceOp.SUM)
    return grad
