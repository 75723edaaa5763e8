"""Multi-process sharding of counts (CPU, gloo, world size 2).

Every rank counts its own row range with the oracle and the ranks sum their
tables; the sum must equal the oracle's tables over the whole database.  A
query split needs no exchange: the ranks' query ranges must tile the batch,
and the slices bench.py hands to its ranks, answered rank by rank and
gathered, must equal the whole batch answered at once.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1804_04640_gb300 import shard

WORLD = 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import oracle
    from workloads import random_dag_database, random_queries

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        db = random_dag_database(9, 20_000 + 123, 2, 5, 3, 0.5, seed=77)
        lo, hi = shard.row_range(db.m, rank, world)
        part = oracle.DB(db.D[:, lo:hi], db.arities)
        queries = random_queries(db.n, 40, 1, 5, seed=78)
        tables = np.concatenate([part.table(q) for q in queries])
        total = shard.allreduce_tables(tables)
        if rank == 0:
            full = oracle.DB(db.D, db.arities)
            want = np.concatenate([full.table(q) for q in queries])
            out.put(bool(np.array_equal(total, want)))
    finally:
        dist.destroy_process_group()


def _query_worker(rank, world, port, out):
    import sys

    import torch.distributed as dist

    import oracle

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # the batch split exactly as the benchmark splits it over its ranks
        w = bench.make_workload("random", m=20_000, nq=60, rank=rank, world=world)
        orc = oracle.DB(w["db"].D, w["db"].arities)
        mine = [orc.table(q) for q in w["queries"]]
        parts = [None] * world
        dist.all_gather_object(parts, (w["queries"], mine))
        if rank == 0:
            whole = bench.make_workload("random", m=20_000, nq=60 * world)
            got_q = [q for p in parts for q in p[0]]
            got_t = [t for p in parts for t in p[1]]
            ok = got_q == whole["queries"] and len(got_t) == len(whole["queries"])
            full = oracle.DB(whole["db"].D, whole["db"].arities)
            ok = ok and all(np.array_equal(t, full.table(q)) for q, t in zip(whole["queries"], got_t))
            ok = ok and all(len(p[0]) == 60 for p in parts)
            out.put(bool(ok))
    finally:
        dist.destroy_process_group()


def test_bench_query_slices_answer_the_whole_batch_once():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_query_worker, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    ok = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert ok


def test_row_shards_sum_to_whole_table():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    ok = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert ok


@pytest.mark.parametrize("m", [1, 4095, 4096, 4097, 100_000])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_ranges_tile_the_work(m, world):
    rows = [shard.row_range(m, r, world) for r in range(world)]
    assert rows[0][0] == 0 and rows[-1][1] == m
    for (a, b), (c, d) in zip(rows, rows[1:]):
        assert b == c and a <= b
    for lo, _ in rows:
        assert lo % shard.CHUNK_ROWS == 0 or lo == m
    qs = [shard.query_range(1000, r, world) for r in range(world)]
    assert qs[0][0] == 0 and qs[-1][1] == 1000
    assert all(b == c for (_, b), (c, _) in zip(qs, qs[1:]))
