"""Tally rows across ranks (one process per GPU, torch.distributed).

Each rank analyses its own trace; the tallies are then one exchange: the
rows of every rank gathered to one rank (the 56-byte row is the exchange
format) and merged there with thapi_tally_merge (exact integer sums, minima
and maxima per (host_id, pid, tid, func_id)).  The gather is host-side
plumbing over whatever process group is given (gloo or NCCL); the merge runs
on the GPU of the receiving rank.
"""
from __future__ import annotations

import numpy as np

from .thapi import ROW_DTYPE


def gather_rows(rows, dst: int = 0, group=None):
    """Every rank's tally rows, concatenated in rank order, on rank ``dst``; None elsewhere."""
    import torch.distributed as dist

    payload = np.ascontiguousarray(rows, dtype=ROW_DTYPE).tobytes()
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    parts = [None] * world if rank == dst else None
    dist.gather_object(payload, parts, dst=dst, group=group)
    if rank != dst:
        return None
    return np.concatenate([np.frombuffer(p, dtype=ROW_DTYPE) for p in parts]) if parts else np.zeros(0, ROW_DTYPE)


def merged_tally(ctx, rows, dst: int = 0, group=None):
    """gather_rows, then thapi_tally_merge on rank ``dst`` (None elsewhere)."""
    from .thapi import thapi_tally_merge

    allrows = gather_rows(rows, dst, group)
    if allrows is None:
        return None
    return thapi_tally_merge(ctx.handle if hasattr(ctx, "handle") else ctx, allrows)
