"""GPU parity of counting queries (C ABI) against the CPU oracle.

Counts must match bit-exactly, for every strategy, at sizes that span several
4096-row work granules with a ragged tail, at the full sizes of the tiny and
batched-random workloads, and on the edge cases of the method.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
import paper_1804_04640_gb300 as fc
from workloads import CONFIGS, config_database, random_dag_database, random_queries, subset_queries

pytestmark = pytest.mark.gpu

STRATS = [fc.FC_STRAT_BITMAP, fc.FC_STRAT_HIST, fc.FC_STRAT_GATOMIC, fc.FC_STRAT_SORT, fc.FC_STRAT_WINDOW]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fc.load_library(build_if_missing=True)


def oracle_tables(orc, queries):
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return list(ex.map(orc.table, queries))


def check_batch(ctx, orc, queries, want=None):
    off, flat = fc.pack_lists(queries)
    tables, toff = fc.fc_count_batch(ctx, off, flat)
    if want is None:
        want = oracle_tables(orc, queries)
    for q, w in enumerate(want):
        got = tables[toff[q]:toff[q + 1]].astype(np.int64)
        assert np.array_equal(got, w), f"query {q} {queries[q]}"
    return want


def test_tiny_all_92_queries():
    """Tiny workload: n=8, m=1000, all 92 subsets of size 1-3."""
    db = config_database("tiny")
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    queries = subset_queries(db.n, (1, 2, 3))
    assert len(queries) == 92
    want = check_batch(ctx, orc, queries)
    for s in STRATS:
        fc.fc_set_option(ctx, "strategy", s)
        check_batch(ctx, orc, queries, want)
    fc.fc_set_option(ctx, "strategy", fc.FC_STRAT_AUTO)
    for q in queries[::7]:                       # single-query entry point
        assert np.array_equal(fc.fc_count(ctx, q).astype(np.int64), orc.table(q))


def test_random_full_size_all_queries():
    """Batched random workload at full size: 10,000 queries, m = 100,000."""
    c = CONFIGS["random"]
    db = config_database("random")
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    queries = random_queries(db.n, c["nq"], c["k"][0], c["k"][1], c["seed"])
    want = check_batch(ctx, orc, queries)
    sub = queries[::25]
    for s in STRATS:
        fc.fc_set_option(ctx, "strategy", s)
        check_batch(ctx, orc, sub, want[::25])


@pytest.mark.parametrize("m", [1, 17, 63, 64, 65, 511, 513, 1023, 1025, 4095, 4096, 4097, 70_001, 131_072 + 13])
def test_ragged_sizes_every_strategy(m):
    db = random_dag_database(9, m, 2, 5, 3, 0.5, seed=1000 + m % 97)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    queries = random_queries(db.n, 60, 1, 6, seed=m) + [[0], [8, 3]]
    want = oracle_tables(orc, queries)
    for s in [fc.FC_STRAT_AUTO] + STRATS:
        fc.fc_set_option(ctx, "strategy", s)
        check_batch(ctx, orc, queries, want)
    fc.fc_set_option(ctx, "strategy", fc.FC_STRAT_HIST)
    fc.fc_set_option(ctx, "smem_cells", 40_000)        # interleaved table copies change
    check_batch(ctx, orc, queries, want)


def test_row_split_work_items():
    """Few queries over many rows: the planner splits rows across CTAs and
    the partial tables are summed in global memory."""
    db = random_dag_database(10, 600_000 + 77, 2, 4, 3, 0.5, seed=5)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    queries = [[0, 1], [2, 3, 4], [5], [9, 8, 7, 6]]
    want = oracle_tables(orc, queries)
    for s in [fc.FC_STRAT_AUTO] + STRATS:
        fc.fc_set_option(ctx, "strategy", s)
        check_batch(ctx, orc, queries, want)


def test_large_tables_sort_and_global_paths():
    """Tables above the shared-memory threshold (up to 16^5 cells)."""
    db = random_dag_database(8, 300_001, 12, 16, 2, 0.3, seed=9)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    queries = [[0, 1, 2, 3, 4], [5, 6, 7, 0], [1, 2, 3]]
    want = oracle_tables(orc, queries)
    check_batch(ctx, orc, queries, want)
    for s in (fc.FC_STRAT_GATOMIC, fc.FC_STRAT_SORT, fc.FC_STRAT_WINDOW):
        fc.fc_set_option(ctx, "strategy", s)
        check_batch(ctx, orc, queries, want)
    fc.fc_set_option(ctx, "strategy", fc.FC_STRAT_AUTO)
    fc.fc_set_option(ctx, "sort_min_cells", 1000)      # route big tables to sort
    check_batch(ctx, orc, queries, want)
    fc.fc_set_option(ctx, "smem_cells", 256)           # everything leaves shared memory
    check_batch(ctx, orc, queries, want)


def test_window_path_cuts_and_row_splits():
    """Tables beyond shared memory counted window by window: the planner's
    choice, uneven last windows, many windows per table, windows whose rows
    are split over several CTAs (few queries), and scores over windowed
    tables."""
    db = random_dag_database(8, 250_003, 12, 16, 2, 0.3, seed=19)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    queries = [[0, 1, 2, 3, 4], [5, 6, 7, 0], [1, 2, 3], [7, 6, 5, 4, 3]]
    want = oracle_tables(orc, queries)
    off, flat = fc.pack_lists(queries)
    plan = fc.fc_plan_count(ctx, off, flat)
    strat = fc.fc_plan_strategies(plan)
    fc.fc_plan_free(plan)
    cells = [int(np.prod([db.arities[v] for v in q])) for q in queries]
    assert all(s == fc.FC_STRAT_WINDOW for s, n in zip(strat, cells) if 24576 < n <= 16 * 50_000)
    check_batch(ctx, orc, queries, want)
    fc.fc_set_option(ctx, "strategy", fc.FC_STRAT_WINDOW)
    for wide in (1, 0):                                # own launch / inside the mixed launch
        fc.fc_set_option(ctx, "window_wide", wide)
        for cells_per_window in (1 << 20, 7001, 1000):  # as many as fit .. ~1000 windows per table
            fc.fc_set_option(ctx, "window_cells", cells_per_window)
            check_batch(ctx, orc, queries, want)
            check_batch(ctx, orc, queries[:1], want[:1])   # one query: rows split per window
    # windowed and shared-memory queries in one plan (two launches)
    fc.fc_set_option(ctx, "window_wide", 1)
    fc.fc_set_option(ctx, "strategy", fc.FC_STRAT_AUTO)
    mixed = queries + [[0, 1], [2, 5, 6], [7]]
    check_batch(ctx, orc, mixed, want + oracle_tables(orc, mixed[len(queries):]))
    with pytest.raises(fc.FcError):
        fc.fc_set_option(ctx, "strategy", fc.FC_STRAT_MARGINAL)   # planner-only strategy
    # a score over a windowed table (its table lives in global memory)
    child, parents = 4, [0, 1, 2, 3]
    fc.fc_set_option(ctx, "strategy", fc.FC_STRAT_WINDOW)
    fc.fc_set_option(ctx, "window_cells", 7001)
    for kind in ("ll", "bdeu"):
        po, pa = fc.pack_lists([parents])
        got = fc.fc_score_batch(ctx, [child], po, pa, kind, ess=1.0)[0]
        ref = orc.score(child, parents, kind, 1.0)
        assert abs(got - ref) <= 1e-5 * max(1.0, abs(ref)), (kind, got, ref)


def test_launch_shape_follows_table_sizes():
    """The planner's two launch shapes: small CTAs unless enough tables need
    more shared memory than they hold; tables beyond the small shape in a
    batch that takes it are planned again (windows or bitmaps)."""
    db = random_dag_database(12, 40_009, 5, 5, 3, 1.0, seed=29)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    rng = np.random.default_rng(30)
    big = [[int(x) for x in rng.choice(db.n, size=6, replace=False)] for _ in range(40)]   # 15,625 cells
    small = random_queries(db.n, 4000, 1, 3, seed=31)
    for queries, big_on_hist in ((big, True), (big + small, False)):
        off, flat = fc.pack_lists(queries)
        plan = fc.fc_plan_count(ctx, off, flat)
        strat = fc.fc_plan_strategies(plan)[:len(big)]
        fc.fc_plan_free(plan)
        if big_on_hist:
            assert (strat != fc.FC_STRAT_WINDOW).all()
        else:
            assert (strat != fc.FC_STRAT_HIST).all()
        sample = big + queries[len(big)::97]
        want = oracle_tables(orc, sample)
        tables, toff = fc.fc_count_batch(ctx, off, flat)
        for i, q in enumerate(list(range(len(big))) + list(range(len(big), len(queries), 97))):
            assert np.array_equal(tables[toff[q]:toff[q + 1]].astype(np.int64), want[i]), q


def test_window_digits_paired_and_single():
    """Windowed keys with neighbouring variables paired into byte digits
    (joint arity <= 256), left single (joint arity > 256), and mixed."""
    db = random_dag_database(8, 90_017, 12, 40, 2, 0.5, seed=37)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    ar = db.arities
    small = [v for v in range(db.n) if ar[v] <= 16]
    big = [v for v in range(db.n) if ar[v] > 16]
    queries = [list(range(db.n))[:3], list(range(db.n))[3:6], list(range(db.n))[5:8]]
    if len(small) >= 2 and big:
        queries += [small[:2] + big[:1], big[:1] + small[:2]]
    if len(big) >= 3:
        queries.append(big[:3])
    want = oracle_tables(orc, queries)
    fc.fc_set_option(ctx, "strategy", fc.FC_STRAT_WINDOW)
    for cells_per_window in (1 << 20, 5003):
        fc.fc_set_option(ctx, "window_cells", cells_per_window)
        check_batch(ctx, orc, queries, want)


def test_edge_cases():
    D = np.array([[0, 1, 0, 1, 1], [0, 0, 0, 0, 0], [2, 1, 0, 2, 2]], dtype=np.uint8)
    ar = [2, 1, 3]
    ctx = fc.fc_load(D, ar)
    orc = oracle.DB(D, ar)
    assert fc.fc_count(ctx, []).tolist() == [5]                    # k = 0: the single cell m
    assert fc.fc_count(ctx, [1]).tolist() == [5]                   # arity-1 variable
    for q in ([1, 0], [0, 1, 2], [2, 1], [2, 0, 1]):
        assert np.array_equal(fc.fc_count(ctx, q).astype(np.int64), orc.table(q))
    with pytest.raises(fc.FcError) as e:
        fc.fc_count(ctx, [0, 0])                                   # duplicate variable
    assert e.value.code == fc.FC_ERR_ARG
    with pytest.raises(fc.FcError) as e:
        fc.fc_count(ctx, [3])                                      # out of range
    assert e.value.code == fc.FC_ERR_ARG
    with pytest.raises(fc.FcError) as e:
        fc.fc_load(np.array([[0, 2]], dtype=np.uint8), [2])        # state >= arity
    assert e.value.code == fc.FC_ERR_RANGE
    big = fc.fc_load(np.zeros((9, 3), dtype=np.uint8), [255] * 9)
    with pytest.raises(fc.FcError) as e:
        fc.fc_count(big, list(range(9)))                           # 255^9 cells
    assert e.value.code == fc.FC_ERR_SIZE
    # empty batch
    tables, toff = fc.fc_count_batch(ctx, np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32))
    assert toff.tolist() == [0]


def test_large_batch_validation_errors():
    """Batches large enough to be planned on several host threads report the
    first invalid query with its own message, and a valid batch of the same
    size still matches the oracle."""
    db = random_dag_database(12, 5003, 2, 4, 3, 1.0, seed=19)
    ctx = fc.fc_load(db.D, db.arities)
    queries = random_queries(db.n, 9000, 1, 4, seed=20)
    bad = [list(q) for q in queries]
    bad[6100] = [0, 99]
    bad[7000] = [3, 3]
    with pytest.raises(fc.FcError) as e:
        fc.fc_count_batch(ctx, *fc.pack_lists(bad))
    assert e.value.code == fc.FC_ERR_ARG and "99" in str(e.value)
    bad[6100] = [0, 1]
    with pytest.raises(fc.FcError) as e:
        fc.fc_count_batch(ctx, *fc.pack_lists(bad))
    assert e.value.code == fc.FC_ERR_ARG and "twice" in str(e.value)
    off, flat = fc.pack_lists(queries)
    tables, toff = fc.fc_count_batch(ctx, off, flat)
    orc = oracle.DB(db.D, db.arities)
    for q in range(0, len(queries), 97):
        assert np.array_equal(tables[toff[q]:toff[q + 1]].astype(np.int64), orc.table(queries[q]))
    child = [q[-1] for q in queries]
    po, pa = fc.pack_lists([q[:-1] for q in queries])
    s1 = fc.fc_score_batch(ctx, child, po, pa, "mdl")
    for q in range(0, len(queries), 211):
        w = orc.score(child[q], queries[q][:-1], "mdl")
        assert abs(float(s1[q]) - w) <= 1e-5 * abs(w) + 1e-12


def test_two_half_batches_offsets_and_errors():
    """Batches of 4096+ queries run in two halves (the second planned while
    the first runs): padded caller offsets, packed offsets (table_off NULL
    through the C ABI), and a bad offset in the second half reported with its
    query's index in the whole batch."""
    db = random_dag_database(14, 30_011, 2, 4, 3, 1.0, seed=23)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    queries = random_queries(db.n, 6001, 1, 5, seed=24)
    off, flat = fc.pack_lists(queries)
    cells = np.array([int(np.prod([db.arities[v] for v in q])) for q in queries], dtype=np.int64)
    padded = np.zeros(len(queries) + 1, dtype=np.int64)
    padded[1:] = np.cumsum(cells + 3)
    tables, _ = fc.fc_count_batch(ctx, off, flat, padded)
    for q in range(0, len(queries), 37):
        assert np.array_equal(tables[padded[q]:padded[q] + cells[q]].astype(np.int64), orc.table(queries[q]))
    lib = fc.load_library()
    packed = np.zeros(int(cells.sum()), dtype=np.int32)
    rc = lib.fc_count_batch(ctx.ptr, len(queries), fc._ptr(off, fc._i32p), fc._ptr(flat, fc._i32p), None,
                            fc._ptr(packed))
    assert rc == fc.FC_OK, fc.fc_last_error()
    dense = np.concatenate([[0], np.cumsum(cells)])
    for q in range(3, len(queries), 41):
        assert np.array_equal(packed[dense[q]:dense[q + 1]], tables[padded[q]:padded[q] + cells[q]])
    short = padded.copy()
    short[4001:] -= cells[4000] + 3 - 1                 # query 4000 gets one cell
    if cells[4000] > 1:
        with pytest.raises(fc.FcError) as e:
            fc.fc_count_batch(ctx, off, flat, short)
        assert e.value.code == fc.FC_ERR_ARG and "query 4000 " in str(e.value)


def test_row_major_load_and_assignment_count():
    """fc_load with a row-major database; Count of a specific assignment
    (the worked example of Sec. 2 lives in tests/golden)."""
    rows = [[int(x) for x in line.split()] for line in open(
        os.path.join(os.path.dirname(__file__), "golden", "worked_example.txt"))
        if line.strip() and line[0].isdigit()]
    R = np.array(rows, dtype=np.uint8) - 1                     # (m, n), 0-based
    ctx = fc.fc_load(R, [3, 2, 2], layout=fc.FC_ROW_MAJOR)
    assert fc.fc_count_assignment(ctx, [0, 1, 2], [2, 1, 0]) == 2
    orc = oracle.DB(R.T, [3, 2, 2])
    for q in ([0], [2, 0], [1, 2, 0]):
        assert np.array_equal(fc.fc_count(ctx, q).astype(np.int64), orc.table(q))
    db = random_dag_database(7, 50_001, 2, 4, 2, 0.5, seed=3)
    ctx2 = fc.fc_load(db.D, db.arities)
    orc2 = oracle.DB(db.D, db.arities)
    rng = np.random.default_rng(0)
    for _ in range(20):
        k = int(rng.integers(1, 5))
        vs = [int(x) for x in rng.choice(7, size=k, replace=False)]
        st = [int(rng.integers(0, db.arities[v])) for v in vs]
        assert fc.fc_count_assignment(ctx2, vs, st) == orc2.count_assignment(vs, st)
    assert fc.fc_count_assignment(ctx2, [0], [200]) == 0


def test_plan_graph_replay_on_stream_is_deterministic():
    torch = pytest.importorskip("torch")
    db = config_database("random")
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    queries = random_queries(db.n, 2000, 2, 6, seed=77)
    off, flat = fc.pack_lists(queries)
    plan = fc.fc_plan_count(ctx, off, flat)
    toff = fc.fc_plan_table_offsets(plan)
    out = torch.zeros(int(toff[-1]), dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    results = []
    for _ in range(3):
        out.fill_(-7)
        s.wait_stream(torch.cuda.current_stream())
        fc.fc_plan_run(plan, out, stream=s)
        fc.fc_sync(ctx, s)
        results.append(out.cpu().numpy().copy())
    assert all(np.array_equal(results[0], r) for r in results[1:])
    want = oracle_tables(orc, queries)
    for q, w in enumerate(want):
        assert np.array_equal(results[0][toff[q]:toff[q + 1]].astype(np.int64), w)
    strat = fc.fc_plan_strategies(plan)
    assert set(np.unique(strat)) <= {fc.FC_STRAT_BITMAP, fc.FC_STRAT_HIST, fc.FC_STRAT_WINDOW}
    # windows only for tables beyond the shared-memory table area of the launch
    cells = np.array([int(np.prod([db.arities[v] for v in q])) for q in queries])
    assert (cells[strat == fc.FC_STRAT_WINDOW] > 8192).all()


def test_bounded_wait_reports_timeout_and_context_survives():
    db = random_dag_database(5, 10_000, 2, 3, 2, 0.5, seed=8)
    ctx = fc.fc_load(db.D, db.arities)
    assert fc.fc_selftest_wait_timeout(ctx, 2000) == fc.FC_ERR_TIMEOUT
    orc = oracle.DB(db.D, db.arities)
    assert np.array_equal(fc.fc_count(ctx, [0, 1]).astype(np.int64), orc.table([0, 1]))
    fc.fc_sync(ctx)                                            # status was cleared


def test_batch_autotuner_keeps_counts_exact():
    db = random_dag_database(20, 60_001, 2, 5, 3, 0.5, seed=61)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    queries = random_queries(db.n, 1500, 1, 6, seed=62)
    off, flat = fc.pack_lists(queries)
    fc.fc_autotune_batch(ctx, off, flat)
    assert fc.fc_get_option(ctx, "bitmap_cost") > 0
    check_batch(ctx, orc, queries)


@pytest.mark.parametrize("m", [1, 100, 70_001, 1_000_003])
def test_assignment_batch(m):
    """Batched specific assignments (end of Sec. 3.3) against the oracle's
    row-by-row Count, with out-of-range states, repeated variables and empty
    assignments."""
    db = random_dag_database(12, m, 2, 5, 3, 0.5, seed=71)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    rng = np.random.default_rng(m)
    qs = []
    for _ in range(3000):
        k = int(rng.integers(0, 9))
        vs = [int(x) for x in rng.choice(db.n, size=k, replace=False)]
        st = [int(rng.integers(0, db.arities[v])) for v in vs]
        qs.append((vs, st))
    qs += [([3], [7]), ([2, 2], [0, 0]), ([2, 2], [0, 1]), ([], []), ([5, 1], [0, 200])]
    vo, vv = fc.pack_lists([q[0] for q in qs])
    _, ss = fc.pack_lists([q[1] for q in qs])
    got = fc.fc_count_assignment_batch(ctx, vo, vv, ss)
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        want = list(ex.map(lambda q: orc.count_assignment(*q), qs))
    assert got.tolist() == want


def test_contexts_on_concurrent_host_threads():
    """Two contexts driven from two host threads at once (ctypes drops the
    GIL): the shared launch-attribute and occupancy caches are thread-safe and
    every result matches a single-threaded run."""
    import threading
    dbs = [random_dag_database(14, 30_001 + 7 * t, 2, 5, 3, 1.0, seed=60 + t) for t in range(2)]
    qs = [random_queries(14, 5000, 1, 5, seed=70 + t) for t in range(2)]
    want = []
    for db, q in zip(dbs, qs):
        ctx = fc.fc_load(db.D, db.arities)
        want.append(fc.fc_count_batch(ctx, *fc.pack_lists(q))[0])
    got = [None, None]
    errors = []

    def run(t):
        try:
            ctx = fc.fc_load(dbs[t].D, dbs[t].arities)
            off, flat = fc.pack_lists(qs[t])
            for _ in range(3):
                got[t] = fc.fc_count_batch(ctx, off, flat)[0]
        except Exception as e:  # noqa: BLE001
            errors.append(e)

    th = [threading.Thread(target=run, args=(t,)) for t in range(2)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errors, errors
    for t in range(2):
        assert np.array_equal(got[t], want[t])


@pytest.mark.parametrize("nq", [300, 6001])
def test_pinned_outputs_are_written_by_the_kernels(nq):
    """A page-locked output buffer whose plan only stores its cells is written
    by the kernels directly (zero_copy); the tables and scores equal those of
    the copied path (a numpy buffer, and zero_copy off), also with padded
    caller offsets, and a batch that accumulates (forced bitmap strategy)
    falls back to the copy.  Both the one-part and the
    two-part (>= 4096 queries) calls are covered."""
    torch = pytest.importorskip("torch")
    db = random_dag_database(16, 50_003, 2, 5, 3, 0.5, seed=61)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    queries = random_queries(db.n, nq, 1, 5, seed=62)
    off, flat = fc.pack_lists(queries)
    copied, toff = fc.fc_count_batch(ctx, off, flat)
    for q in range(0, nq, max(1, nq // 60)):
        assert np.array_equal(copied[toff[q]:toff[q + 1]].astype(np.int64), orc.table(queries[q]))
    pinned = torch.full((int(toff[-1]),), -9, dtype=torch.int32).pin_memory()
    fc.fc_count_batch(ctx, off, flat, toff, out=pinned)
    assert np.array_equal(pinned.numpy(), copied[: int(toff[-1])])
    # padded offsets (the cells between tables are unspecified)
    cells = np.diff(toff)
    padded = np.zeros(nq + 1, dtype=np.int64)
    padded[1:] = np.cumsum(cells + 2)
    pad_out = torch.full((int(padded[-1]),), -9, dtype=torch.int32).pin_memory()
    fc.fc_count_batch(ctx, off, flat, padded, out=pad_out)
    got = pad_out.numpy()
    for q in range(nq):
        assert np.array_equal(got[padded[q]:padded[q] + cells[q]], copied[toff[q]:toff[q + 1]])
    # scores into a page-locked buffer equal the copied ones
    child = [q[0] for q in queries]
    po, pa = fc.pack_lists([q[1:] for q in queries])
    s_copy = fc.fc_score_batch(ctx, child, po, pa, "bdeu", 1.0)
    s_pin = torch.zeros(nq, dtype=torch.float32).pin_memory()
    fc.fc_score_batch(ctx, child, po, pa, "bdeu", 1.0, out=s_pin)
    assert np.array_equal(s_pin.numpy(), s_copy[:nq])
    # zero_copy off, and an accumulating plan, take the copy path
    fc.fc_set_option(ctx, "zero_copy", 0)
    off_out = torch.full((int(toff[-1]),), -9, dtype=torch.int32).pin_memory()
    fc.fc_count_batch(ctx, off, flat, toff, out=off_out)
    assert np.array_equal(off_out.numpy(), copied[: int(toff[-1])])
    fc.fc_set_option(ctx, "zero_copy", 1)
    fc.fc_set_option(ctx, "strategy", fc.FC_STRAT_BITMAP)
    bm_out = torch.full((int(toff[-1]),), -9, dtype=torch.int32).pin_memory()
    fc.fc_count_batch(ctx, off, flat, toff, out=bm_out)
    assert np.array_equal(bm_out.numpy(), copied[: int(toff[-1])])


def test_device_planned_batches_match_host_planned():
    """Batches of 4096+ queries whose queries all count in shared memory are
    planned on the device (option device_plan).  Their tables equal the host
    planner's (device_plan off) and the oracle's, with caller offsets or
    packed, into numpy or page-locked buffers; a batch the fast path does not
    take (a forced bitmap strategy, a table beyond the mixed launch's
    windows) and an invalid batch go to the host planner, which reports the
    error with the failing query's index."""
    torch = pytest.importorskip("torch")
    db = random_dag_database(40, 60_011, 2, 5, 3, 0.5, seed=71)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    queries = random_queries(db.n, 6000, 1, 6, seed=72)
    off, flat = fc.pack_lists(queries)
    # a cost model under which no query prefers the bitmap strategy (as the
    # autotuner sets it on this kind of batch): the fast path's condition
    for key in ("bitmap_cost", "bitmap_chunk_cost", "small_cost", "small3_cost"):
        fc.fc_set_option(ctx, key, 10 ** 9)
    fc.fc_set_option(ctx, "device_plan", 0)
    host_t, toff = fc.fc_count_batch(ctx, off, flat)
    assert fc.fc_info(ctx, 7) == 0
    fc.fc_set_option(ctx, "device_plan", 1)
    dev_t, toff2 = fc.fc_count_batch(ctx, off, flat)
    assert fc.fc_info(ctx, 7) == 1
    assert np.array_equal(toff, toff2)
    assert np.array_equal(dev_t, host_t)
    for q in range(0, len(queries), 97):
        assert np.array_equal(dev_t[toff[q]:toff[q + 1]].astype(np.int64), orc.table(queries[q]))
    # caller offsets (padded), numpy and page-locked outputs
    cells = np.diff(toff)
    padded = np.zeros(len(queries) + 1, dtype=np.int64)
    padded[1:] = np.cumsum(cells + 1)
    for pin in (False, True):
        out = torch.full((int(padded[-1]),), -3, dtype=torch.int32)
        if pin:
            out = out.pin_memory()
        fc.fc_count_batch(ctx, off, flat, padded, out=out if pin else out.numpy())
        assert fc.fc_info(ctx, 7) == 1
        got = out.numpy()
        for q in range(len(queries)):
            assert np.array_equal(got[padded[q]:padded[q] + cells[q]], host_t[toff[q]:toff[q + 1]])
    # the caller's lists in page-locked memory
    p_off = torch.from_numpy(np.ascontiguousarray(off, dtype=np.int32)).pin_memory()
    p_flat = torch.from_numpy(np.ascontiguousarray(flat, dtype=np.int32)).pin_memory()
    p_to = torch.from_numpy(np.ascontiguousarray(padded, dtype=np.int64)).pin_memory()
    for pin_out in (False, True):
        out = torch.full((int(padded[-1]),), -5, dtype=torch.int32)
        if pin_out:
            out = out.pin_memory()
        fc.fc_count_batch(ctx, p_off, p_flat, p_to, out=out if pin_out else out.numpy())
        assert fc.fc_info(ctx, 7) == 1
        got = out.numpy()
        for q in range(len(queries)):
            assert np.array_equal(got[padded[q]:padded[q] + cells[q]], host_t[toff[q]:toff[q + 1]])
    # packed offsets through the C ABI (table_off NULL)
    lib = fc.load_library()
    packed = np.zeros(int(toff[-1]), dtype=np.int32)
    rc = lib.fc_count_batch(ctx.ptr, len(queries), fc._ptr(off, fc._i32p), fc._ptr(flat, fc._i32p), None,
                            fc._ptr(packed))
    assert rc == fc.FC_OK, fc.fc_last_error()
    assert fc.fc_info(ctx, 7) == 1
    assert np.array_equal(packed, host_t[: int(toff[-1])])
    # the host planner takes batches the fast path does not: a forced bitmap
    # strategy, and a table beyond the small shape's windows
    fc.fc_set_option(ctx, "strategy", fc.FC_STRAT_BITMAP)
    bm_t, _ = fc.fc_count_batch(ctx, off, flat)
    assert fc.fc_info(ctx, 7) == 0
    assert np.array_equal(bm_t, host_t)
    fc.fc_set_option(ctx, "strategy", fc.FC_STRAT_AUTO)
    wide = list(queries)
    big = sorted(range(db.n), key=lambda v: -int(db.arities[v]))[:9]   # > 16384 cells
    wide[17] = big
    o3, f3 = fc.pack_lists(wide)
    w_t, wto = fc.fc_count_batch(ctx, o3, f3)
    assert fc.fc_info(ctx, 7) == 0
    assert np.array_equal(w_t[wto[17]:wto[18]].astype(np.int64), orc.table(big))
    assert np.array_equal(w_t[wto[18]:wto[19]], host_t[toff[18]:toff[19]])
    # an invalid query: the host planner's error, with its index
    bad = list(queries)
    bad[4500] = [0, db.n + 3]
    ob, fb = fc.pack_lists(bad)
    with pytest.raises(fc.FcError) as e:
        fc.fc_count_batch(ctx, ob, fb)
    assert e.value.code == fc.FC_ERR_ARG and "out of range" in str(e.value)
    # the context still answers after the refused batch
    again, _ = fc.fc_count_batch(ctx, off, flat)
    assert np.array_equal(again, host_t)


@pytest.mark.parametrize("m,ar", [(4096 * 3 + 17, [16, 2, 3, 16, 5, 1, 7, 16, 4]),
                                  (40_000, [16, 2, 3, 16, 5, 1, 7, 16, 4]),
                                  (4096 * 5 + 999, [4, 2, 3, 4, 4, 1, 2, 3, 4])])
def test_codes4_matches_byte_columns(m, ar):
    """On a database whose arities are all <= 16 the histogram strategy reads
    the 4-bit copy of the columns (option codes4).  Its tables equal the byte
    columns' and the oracle's: arity 16 (the top code 15 in a nibble), arity
    1, ragged tails that end inside a 32-row group, the copy repacked by
    appends that start at odd rows, and (all arities <= 4) the keys that pair
    variables on the packed nibbles."""
    rng = np.random.default_rng(m)
    n = 9
    ar = np.array(ar, dtype=np.int32)
    D = np.stack([rng.integers(0, a, size=m) for a in ar]).astype(np.uint8)
    D[0, -1] = ar[0] - 1
    D[3, :50] = ar[3] - 1
    queries = random_queries(n, 400, 1, 6, seed=m + 1) + [[0, 3], [0, 3, 7], [5], [5, 0], list(range(6))]
    queries = [q for q in queries if int(np.prod(ar[q])) <= 16384]
    ctx = fc.fc_load(D, ar)
    assert fc.fc_info(ctx, 6) == 4
    fc.fc_set_option(ctx, "strategy", fc.FC_STRAT_HIST)
    for cut in (0, 1, 33):
        if cut:
            extra = np.stack([rng.integers(0, a, size=cut * 7 + 3) for a in ar]).astype(np.uint8)
            fc.fc_append(ctx, extra)
            D = np.concatenate([D, extra], axis=1)
        orc = oracle.DB(D, ar)
        off, flat = fc.pack_lists(queries)
        fc.fc_set_option(ctx, "codes4", 0)
        byte_t, toff = fc.fc_count_batch(ctx, off, flat)
        fc.fc_set_option(ctx, "codes4", 1)
        nib_t, toff2 = fc.fc_count_batch(ctx, off, flat)
        assert np.array_equal(toff, toff2)
        assert np.array_equal(nib_t, byte_t)
        for q in range(0, len(queries), 7):
            assert np.array_equal(nib_t[toff[q]:toff[q + 1]].astype(np.int64), orc.table(queries[q])), queries[q]
        for q in range(len(queries) - 5, len(queries)):
            assert np.array_equal(nib_t[toff[q]:toff[q + 1]].astype(np.int64), orc.table(queries[q])), queries[q]


def test_codes4_only_for_arities_up_to_16():
    """An arity of 17 keeps the byte columns (fc_info key 6 = 8 bits), with
    the same tables as the oracle; switching the option off does the same on
    a database that has the 4-bit copy."""
    rng = np.random.default_rng(5)
    ar = np.array([17, 3, 4], dtype=np.int32)
    D = np.stack([rng.integers(0, a, size=9001) for a in ar]).astype(np.uint8)
    ctx = fc.fc_load(D, ar)
    assert fc.fc_info(ctx, 6) == 8
    orc = oracle.DB(D, ar)
    check_batch(ctx, orc, [[0, 1], [1, 2], [0, 1, 2], [2, 0]])
    ctx2 = fc.fc_load(D[1:], ar[1:])
    assert fc.fc_info(ctx2, 6) == 4
    fc.fc_set_option(ctx2, "codes4", 0)
    assert fc.fc_info(ctx2, 6) == 8
