"""Multi-process helpers for scanning on several GPUs (one process per GPU).

The scan needs no data exchange: a long text is cut into contiguous ranges
of start positions, one per rank; each rank also reads the next
(longest pattern - 1) bytes so that walks starting near its range's end can
finish (the chunk-overlap rule of Section II-B), and its ids are a disjoint
slice of the whole. The only exchange is the sum of the per-rank match
counts (8 bytes). Batches shard by text, balanced by bytes. Timing takes the
maximum over ranks.
"""
from __future__ import annotations

import os
from typing import List, Tuple

import numpy as np


def dist_env() -> Tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_text(n: int, max_len: int, rank: int, world: int) -> Tuple[int, int, int]:
    """Start positions [a, b) of rank's share of a text of n bytes, and the
    readable end `limit` = min(n, b + max_len - 1) its walks may reach."""
    a = n * rank // world
    b = n * (rank + 1) // world
    limit = min(n, b + max(max_len - 1, 0))
    return a, b, limit


def shard_texts(offsets, rank: int, world: int) -> Tuple[int, int]:
    """Texts [t0, t1) of rank's share of a batch, contiguous and balanced by
    bytes (offsets: n+1 non-decreasing byte offsets)."""
    off = np.asarray(offsets, dtype=np.int64)
    total = int(off[-1])
    lo = np.searchsorted(off, total * rank // world, side="left")
    hi = np.searchsorted(off, total * (rank + 1) // world, side="left")
    nt = len(off) - 1
    t0 = min(int(lo), nt)
    t1 = nt if rank == world - 1 else min(int(hi), nt)
    return t0, max(t0, t1)


def sum_over_ranks(value: int, device="cpu") -> int:
    """The count exchange: sum an integer over all ranks."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.int64, device=device)
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


def max_over_ranks(value: float, device="cpu") -> float:
    """Step time of the job: the slowest rank's."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_slices(local, world: int) -> List:
    """All ranks' local arrays (for checks; not on the scan's data path)."""
    import torch.distributed as dist
    if not (dist.is_initialized() and world > 1):
        return [local]
    out = [None] * world
    dist.all_gather_object(out, local)
    return out
