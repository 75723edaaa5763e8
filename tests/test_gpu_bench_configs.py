"""Parity in the launch configuration bench.py times, at the full workload sizes.

Each test builds its workload with bench.make_workload, plans it the way the
benchmark does (batch autotuner, device-resident plan, CUDA-graph replay on a
side stream, twice) and compares with the oracle: every table of the
10,000-query batch (also through the end-to-end call the bench times), and
seeded samples (plus properties that hold at any size) for the larger
workloads.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import bench
import oracle
import paper_1804_04640_gb300 as fc

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fc.load_library(build_if_missing=True)


def _pool_map(fn, xs):
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return list(ex.map(fn, xs))


def _replay(plan, outs, torch):
    s = torch.cuda.Stream()
    results = []
    for _ in range(2):
        for o in outs:
            o.fill_(-1) if o.dtype != torch.float32 else o.fill_(float("nan"))
        s.wait_stream(torch.cuda.current_stream())
        fc.fc_plan_run(plan, *outs, stream=s)
        s.synchronize()
        results.append([o.cpu().numpy().copy() for o in outs])
    for a, b in zip(results[0], results[1]):
        assert np.array_equal(a, b, equal_nan=True)
    return results[1]


def test_random_batch_as_benchmarked():
    torch = pytest.importorskip("torch")
    w = bench.make_workload("random")
    db, queries = w["db"], w["queries"]
    ctx = fc.fc_load(db.D, db.arities)
    off, flat = fc.pack_lists(queries)
    fc.fc_autotune_batch(ctx, off, flat)
    plan = fc.fc_plan_count(ctx, off, flat)
    toff = fc.fc_plan_table_offsets(plan)
    (tables,) = _replay(plan, [torch.empty(int(toff[-1]), dtype=torch.int32, device="cuda")], torch)
    orc = oracle.DB(db.D, db.arities)
    want = _pool_map(orc.table, queries)
    for q, t in enumerate(want):
        assert np.array_equal(tables[toff[q]:toff[q + 1]].astype(np.int64), t), q
    # the end-to-end call the bench times: host lists, planned on the device
    # when the tuned cost model keeps every query in shared memory (the bench
    # line's e2e.planner says which), tables stored straight into a
    # page-locked buffer, twice in a row
    pinned = torch.empty(int(toff[-1]), dtype=torch.int32).pin_memory()
    for _ in range(2):
        pinned.fill_(-1)
        fc.fc_count_batch(ctx, off, flat, toff, out=pinned)
        got = pinned.numpy()
        for q, t in enumerate(want):
            assert np.array_equal(got[toff[q]:toff[q + 1]].astype(np.int64), t), q


def test_scores_batch_as_benchmarked():
    torch = pytest.importorskip("torch")
    w = bench.make_workload("scores")
    db = w["db"]
    ctx = fc.fc_load(db.D, db.arities)
    fo, ff = fc.pack_lists([list(p) + [c] for p, c in zip(w["parents"], w["child"])])
    fc.fc_autotune_batch(ctx, fo, ff)
    po, pa = fc.pack_lists(w["parents"])
    plan = fc.fc_plan_score(ctx, w["child"], po, pa, "bdeu", 1.0)
    (scores,) = _replay(plan, [torch.empty(len(w["child"]), dtype=torch.float32, device="cuda")], torch)
    orc = oracle.DB(db.D, db.arities)
    idx = np.random.default_rng(17).choice(len(w["child"]), size=800, replace=False)
    want = np.array(_pool_map(lambda q: orc.score(w["child"][q], w["parents"][q], "bdeu", 1.0), idx))
    got = scores[idx].astype(np.float64)
    assert np.all(np.abs(got - want) <= 1e-5 * np.abs(want) + 1e-12)


def test_pairs_as_benchmarked():
    torch = pytest.importorskip("torch")
    w = bench.make_workload("pairs")
    db = w["db"]
    ctx = fc.fc_load(db.D, db.arities)
    plan = fc.fc_plan_pairs(ctx)
    outs = [torch.empty(fc.fc_plan_size(plan, 0), dtype=torch.int32, device="cuda"),
            torch.empty(fc.fc_plan_size(plan, 1), dtype=torch.float32, device="cuda")]
    tables, mi = _replay(plan, outs, torch)
    orc = oracle.DB(db.D, db.arities)
    pairs = [(a, b) for a in range(db.n) for b in range(a + 1, db.n)]
    off = np.zeros(len(pairs) + 1, dtype=np.int64)
    off[1:] = np.cumsum([int(db.arities[a]) * int(db.arities[b]) for a, b in pairs])
    sums = np.add.reduceat(tables.astype(np.int64), off[:-1])
    assert np.all(sums == db.m)                                  # every pair table sums to m
    idx = np.random.default_rng(5).choice(len(pairs), size=200, replace=False)

    def one(p):
        a, b = pairs[p]
        t = orc.table([a, b])
        return t, oracle.score_table(t, int(db.arities[a]), int(db.arities[b]), "mi")

    for p, (t, m) in zip(idx, _pool_map(one, idx)):
        assert np.array_equal(tables[off[p]:off[p + 1]].astype(np.int64), t)
        assert abs(float(mi[p]) - m) <= 1e-5 * abs(m) + 1e-12


def test_support_as_benchmarked():
    torch = pytest.importorskip("torch")
    w = bench.make_workload("support")
    bits, m, sets = w["bits"], w["m"], w["sets"]
    ctx = fc.fc_load_bits(bits, m)
    so, it = fc.pack_lists(sets)
    plan = fc.fc_plan_support(ctx, so, it)
    outs = [torch.empty(len(sets), dtype=torch.int32, device="cuda"),
            torch.empty(len(it), dtype=torch.int32, device="cuda"),
            torch.empty(len(it), dtype=torch.float32, device="cuda")]
    supp, sub, conf = _replay(plan, outs, torch)
    owner = np.repeat(np.arange(len(sets)), np.diff(so))
    # invariants on all 1e6 itemsets: anti-monotone supports, confidences in
    # [0, 1] equal to the float quotient of the reported supports
    assert np.all(supp[owner] <= sub)
    want_conf = np.where(sub > 0, supp[owner].astype(np.float32) / np.maximum(sub, 1).astype(np.float32), 0)
    assert np.array_equal(conf, want_conf.astype(np.float32))
    assert np.all((conf >= 0) & (conf <= 1))
    # exact parity on 32 itemsets against the C oracle's transaction scan ...
    idx = np.random.default_rng(9).choice(len(sets), size=32, replace=False)
    for q, (s, sb, c) in zip(idx, _pool_map(lambda q: oracle.support_rules(bits, m, sets[q]), idx)):
        a, b = so[q], so[q + 1]
        assert supp[q] == s and np.array_equal(sub[a:b].astype(np.int64), sb)
        assert np.allclose(conf[a:b], c, rtol=1e-6, atol=0)
    # ... and on 4,096 more (every size) against the oracle's item-matrix
    # definition, unpacking only the items each itemset names
    from oracle import miner
    rng = np.random.default_rng(10)
    sizes = np.diff(so)
    idx = np.concatenate([rng.choice(np.flatnonzero(sizes == k), size=1024, replace=False)
                          for k in range(2, 6)])

    def one(q):
        S = sets[q]
        X = miner.item_matrix_from_bits(bits[S], m)
        loc = list(range(len(S)))
        return (miner.itemset_support(X, loc),
                [miner.itemset_support(X, loc[:t] + loc[t + 1:]) for t in range(len(S))])

    for q, (s, sb) in zip(idx, _pool_map(one, idx)):
        assert supp[q] == s and sub[so[q]:so[q + 1]].tolist() == sb, q


def test_families_as_benchmarked():
    torch = pytest.importorskip("torch")
    w = bench.make_workload("families")
    db = w["db"]
    ctx = fc.fc_load(db.D, db.arities)
    fams = fc.family_list(w["vars"], w["max_parents"])
    fo, ff = fc.pack_lists([list(f[1]) + [f[0]] for f in fams])
    fc.fc_autotune_batch(ctx, fo, ff)
    plan = fc.fc_plan_families(ctx, w["vars"], w["max_parents"], "bdeu", 1.0)
    assert fc.fc_plan_size(plan, 1) == len(fams)
    (scores,) = _replay(plan, [torch.empty(len(fams), dtype=torch.float32, device="cuda")], torch)
    assert np.all(np.isfinite(scores)) and np.all(scores < 0)
    orc = oracle.DB(db.D, db.arities)
    idx = np.random.default_rng(23).choice(len(fams), size=600, replace=False)
    want = np.array(_pool_map(lambda q: orc.score(fams[q][0], fams[q][1], "bdeu", 1.0), idx))
    got = scores[idx].astype(np.float64)
    assert np.all(np.abs(got - want) <= 1e-5 * np.abs(want) + 1e-12)


def test_rules_as_benchmarked():
    """Full-size mining run: every pair of frequent items is checked against a
    complete pair-count matrix, a sample of larger itemsets against the
    oracle's row scan, and every rule against the reported supports."""
    from oracle import miner
    w = bench.make_workload("rules")
    db = w["db"]
    min_support, min_conf, max_size, _ = w["args"]
    ctx = fc.fc_load(db.D, db.arities)
    r = fc.fc_mine_rules(ctx, *w["args"])
    r2 = fc.fc_mine_rules(ctx, *w["args"])
    for k in ("set_off", "items", "support", "rule_set", "antecedent", "confidence"):
        assert np.array_equal(r[k], r2[k])
    so, it, sp = r["set_off"], r["items"], r["support"]
    sets = [tuple(int(x) for x in it[so[i]:so[i + 1]]) for i in range(len(so) - 1)]
    assert sets == sorted(sets, key=lambda S: (len(S), S)) and max(map(len, sets)) <= max_size
    thr = min_support * db.m
    assert all(float(s) > thr for s in sp)
    X = miner.item_matrix_from_db(db.D, db.arities)
    single = X.sum(axis=1)
    freq1 = [i for i in range(X.shape[0]) if float(single[i]) > thr]
    assert [S for S in sets if len(S) == 1] == [(i,) for i in freq1]
    Xf = X[freq1].astype(np.float32)
    pair = (Xf @ Xf.T).astype(np.int64)  # counts <= 1e6 are exact in float32
    want2 = {(freq1[a], freq1[b]): int(pair[a, b]) for a in range(len(freq1)) for b in range(a + 1, len(freq1))
             if float(pair[a, b]) > thr}
    got2 = {S: int(s) for S, s in zip(sets, sp) if len(S) == 2}
    assert got2 == want2
    big = [i for i, S in enumerate(sets) if len(S) >= 3]
    idx = np.random.default_rng(31).choice(big, size=min(300, len(big)), replace=False)
    want = _pool_map(lambda i: miner.itemset_support(X, sets[i]), idx)
    assert [int(sp[i]) for i in idx] == want
    index = {S: i for i, S in enumerate(sets)}
    rules = {(int(a), int(b)): float(c) for a, b, c in zip(r["rule_set"], r["antecedent"], r["confidence"])}
    for i, S in enumerate(sets):
        k = len(S)
        for t in range(k - 1, -1, -1) if k >= 2 else ():
            mk = ((1 << k) - 1) ^ (1 << t)
            sa = int(sp[index[tuple(S[u] for u in range(k) if mk >> u & 1)]])
            keep = float(sp[i]) > min_conf * float(sa)
            assert ((i, mk) in rules) == keep
            if keep:
                assert rules[(i, mk)] == np.float32(float(sp[i]) / float(sa))
    assert len(rules) == len(r["rule_set"])


def test_tiny_and_large_as_benchmarked():
    """The 92-query tiny batch in full and the large-table batch (global-atomic
    path) sampled, through autotuned, graph-replayed plans."""
    torch = pytest.importorskip("torch")
    for name, sample in (("tiny", None), ("large", 12)):
        w = bench.make_workload(name)
        db, queries = w["db"], w["queries"]
        ctx = fc.fc_load(db.D, db.arities)
        off, flat = fc.pack_lists(queries)
        fc.fc_autotune_batch(ctx, off, flat)
        plan = fc.fc_plan_count(ctx, off, flat)
        toff = fc.fc_plan_table_offsets(plan)
        (tables,) = _replay(plan, [torch.empty(int(toff[-1]), dtype=torch.int32, device="cuda")], torch)
        orc = oracle.DB(db.D, db.arities)
        idx = range(len(queries)) if sample is None else \
            np.random.default_rng(3).choice(len(queries), size=sample, replace=False)
        want = _pool_map(lambda q: orc.table(queries[q]), idx)
        for q, t in zip(idx, want):
            assert np.array_equal(tables[toff[q]:toff[q + 1]].astype(np.int64), t), (name, q)
        for q in range(len(queries)):
            assert int(tables[toff[q]:toff[q + 1]].astype(np.int64).sum()) == db.m


def test_assign_as_benchmarked():
    torch = pytest.importorskip("torch")
    w = bench.make_workload("assign")
    db = w["db"]
    ctx = fc.fc_load(db.D, db.arities)
    vo, vv = fc.pack_lists([q[0] for q in w["assign"]])
    _, ss = fc.pack_lists([q[1] for q in w["assign"]])
    plan = fc.fc_plan_assignments(ctx, vo, vv, ss)
    (counts,) = _replay(plan, [torch.empty(len(w["assign"]), dtype=torch.int32, device="cuda")], torch)
    orc = oracle.DB(db.D, db.arities)
    idx = np.random.default_rng(4).choice(len(w["assign"]), size=2000, replace=False)
    want = _pool_map(lambda q: orc.count_assignment(*w["assign"][q]), idx)
    assert [int(counts[q]) for q in idx] == want


def test_splits_as_benchmarked():
    """All-splits plan at full size: 64 itemsets (16 of each size) exact
    against the item-matrix definition, and invariants on every split."""
    torch = pytest.importorskip("torch")
    from oracle import miner
    w = bench.make_workload("splits")
    bits, m, sets = w["bits"], w["m"], w["sets"]
    ctx = fc.fc_load_bits(bits, m)
    so, it = fc.pack_lists(sets)
    plan = fc.fc_plan_support_splits(ctx, so, it)
    ns = fc.fc_plan_size(plan, 3)
    outs = [torch.empty(len(sets), dtype=torch.int32, device="cuda"),
            torch.empty(ns, dtype=torch.int32, device="cuda"),
            torch.empty(ns, dtype=torch.float32, device="cuda")]
    supp, sub, conf = _replay(plan, outs, torch)
    off = fc.split_offsets(so)
    owner = np.repeat(np.arange(len(sets)), np.diff(off))
    assert np.all(supp[owner] <= sub)
    want_conf = np.where(sub > 0, supp[owner].astype(np.float32) / np.maximum(sub, 1).astype(np.float32), 0)
    assert np.array_equal(conf, want_conf.astype(np.float32))
    sizes = np.diff(so)
    rng = np.random.default_rng(12)
    idx = np.concatenate([rng.choice(np.flatnonzero(sizes == k), size=16, replace=False) for k in range(2, 6)])

    def one(q):
        S = sets[q]
        X = miner.item_matrix_from_bits(bits[S], m)
        k = len(S)
        return (miner.itemset_support(X, list(range(k))),
                [miner.itemset_support(X, [t for t in range(k) if mk >> t & 1]) for mk in range(1, (1 << k) - 1)])

    for q, (s, sb) in zip(idx, _pool_map(one, idx)):
        assert supp[q] == s and sub[off[q]:off[q + 1]].tolist() == sb, q


def test_append_as_benchmarked():
    """The append workload's context after warm-up-sized appends from device
    memory equals one load of the same rows (marginals and a query batch)."""
    torch = pytest.importorskip("torch")
    w = bench.make_workload("append")
    db, m0, B = w["db"], w["m0"], w["block"]
    D = np.ascontiguousarray(db.D)
    ctx = fc.fc_load(D[:, :m0], db.arities)
    fc.fc_reserve(ctx, m0 + 4 * B)
    block = torch.from_numpy(np.ascontiguousarray(D[:, m0:m0 + B])).cuda()
    for _ in range(3):
        fc.fc_append(ctx, block)
    full = np.concatenate([D[:, :m0]] + [D[:, m0:m0 + B]] * 3, axis=1)
    ref = fc.fc_load(full, db.arities)
    assert fc.fc_info(ctx, 1) == full.shape[1]
    assert np.array_equal(fc.fc_marginals(ctx), fc.fc_marginals(ref))
    queries = [[0, 1, 2], [5, 9], [10, 20, 30, 40], [63]]
    off, flat = fc.pack_lists(queries)
    a = fc.fc_count_batch(ctx, off, flat)[0]
    assert np.array_equal(a, fc.fc_count_batch(ref, off, flat)[0])
    orc = oracle.DB(full, db.arities)
    toff = np.concatenate([[0], np.cumsum([int(np.prod([db.arities[v] for v in q])) for q in queries])])
    for q, t in zip(range(len(queries)), _pool_map(lambda q: orc.table(queries[q]), range(len(queries)))):
        assert np.array_equal(a[toff[q]:toff[q + 1]].astype(np.int64), t)
