"""Multi-GPU runs: one process per GPU, each running the prox on its own data.

The single-vector prox does not shard without all-to-all exchanges, so runs
with N GPUs are N independent replicas (weak scaling); batched layouts shard
by segment, contiguous ranges of segments with about equal element counts,
and need no collective on the data path either.  The only collectives are
the ones that time a run: a barrier before and after the timed region and a
max over ranks of the measured time.
"""
from __future__ import annotations

import os

import numpy as np


def env():
    """(rank, world_size, local_rank) from the launcher's environment (1 process when unset)."""
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x: float, device="cpu") -> float:
    """Max of x over all ranks of the default process group (x itself without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def shard_segments(offsets, rank: int, world: int):
    """Contiguous segment range [s0, s1) of `rank`: segment boundaries closest to
    equal shares of the elements (every segment goes to exactly one rank)."""
    off = np.asarray(offsets, dtype=np.int64)
    n_seg = off.shape[0] - 1
    if world <= 1 or n_seg <= 0:
        return 0, n_seg
    total = int(off[-1])
    cut = [0]
    for r in range(1, world):
        target = total * r // world
        s = int(np.searchsorted(off, target, side="left"))
        s = min(max(s, cut[-1]), n_seg)
        cut.append(s)
    cut.append(n_seg)
    return cut[rank], cut[rank + 1]


def job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (ms_max / 1e3)
