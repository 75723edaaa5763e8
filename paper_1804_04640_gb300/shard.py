"""Host-side sharding of counting work over several processes.

Counts are sums over instances, so a database can be split by rows: every
rank counts its own contiguous row range and an integer sum-reduction of the
tables gives the exact tables of the whole database (Sec. 2: a count is the
size of a support set, and disjoint row ranges have disjoint supports).
Independent queries can also be split across ranks with no exchange at all.

Row ranges are cut on the 4096-instance granule of the count kernels so that
every rank's work items stay aligned.
"""
from __future__ import annotations

import numpy as np

CHUNK_ROWS = 4096


def row_range(m: int, rank: int, world: int) -> tuple[int, int]:
    """Rows [lo, hi) of `rank` out of `world`, whole 4096-row chunks except the tail."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    chunks = (m + CHUNK_ROWS - 1) // CHUNK_ROWS
    lo = chunks * rank // world * CHUNK_ROWS
    hi = min(m, chunks * (rank + 1) // world * CHUNK_ROWS)
    return min(lo, m), hi


def query_range(nq: int, rank: int, world: int) -> tuple[int, int]:
    """Queries [lo, hi) of `rank` when independent queries are split."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    return nq * rank // world, nq * (rank + 1) // world


def split_batch(batch, rank: int, world: int):
    """The part of a batch of independent queries that `rank` answers: the
    contiguous slice query_range(len(batch), rank, world).  The parts of all
    ranks tile the batch, so every query is answered exactly once."""
    lo, hi = query_range(len(batch), rank, world)
    return batch[lo:hi]


def allreduce_tables(tables: np.ndarray, group=None) -> np.ndarray:
    """Exact sum of the ranks' partial tables (int64, through torch.distributed)."""
    import torch
    import torch.distributed as dist

    t = torch.from_numpy(np.ascontiguousarray(tables, dtype=np.int64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.numpy()
