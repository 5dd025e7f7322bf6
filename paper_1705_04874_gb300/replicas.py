"""Replica parallelism across GPUs: one process per GPU, each with a full copy
of the velocity model, each simulating its own share of the independent
sources (the paper runs batches of sources for one model on separate GPUs,
Sec. III-A).  There is no data-path collective: ranks exchange only the
timing (max over ranks) and, for superposition, their partial gathers (a sum,
Sec. IV), through torch.distributed on the host.
"""
from __future__ import annotations

import numpy as np


def shard(n_items: int, world: int, rank: int) -> range:
    """Contiguous block of item indices owned by `rank` (sizes differ by at
    most one, lower ranks take the extra ones)."""
    if world < 1 or not 0 <= rank < world or n_items < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(dist, value: float) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value: float) -> float:
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def merge_gathers(dist, gather: np.ndarray) -> np.ndarray:
    """Sum the per-rank partial superposition gathers (each rank superposed
    the events of its own sources) into the full gather on every rank."""
    if dist is None:
        return gather
    import torch
    t = torch.from_numpy(np.ascontiguousarray(gather, dtype=np.float32).copy())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def events_of_rank(src_of_event, sources: range):
    """Indices of the events whose source belongs to this rank, and those
    events' source indices relative to the rank's first source."""
    src = np.asarray(src_of_event)
    sel = np.nonzero((src >= sources.start) & (src < sources.stop))[0]
    return sel, (src[sel] - sources.start).astype(np.int32)
