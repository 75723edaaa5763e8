"""GPU parity of a growing database (Sec. 6: instances appended during
processing update the bitmaps; the radix/histogram path reads D as it stands).

After any sequence of appends every query must equal the oracle on the
concatenated database, and a context grown by appends must give bit-identical
results to one loaded with all instances at once.
"""
import numpy as np
import pytest

import oracle
import paper_1804_04640_gb300 as fc
from oracle import miner
from workloads import basket_transaction_bitmaps, random_dag_database, random_queries

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fc.load_library(build_if_missing=True)


def _all_results(ctx, queries, fams):
    off, flat = fc.pack_lists(queries)
    tables = fc.fc_count_batch(ctx, off, flat)[0]
    po, pa = fc.pack_lists([f[1] for f in fams])
    ch = [f[0] for f in fams]
    scores = {k: fc.fc_score_batch(ctx, ch, po, pa, k, 1.0) for k in ("mdl", "bdeu", "mi")}
    return tables, scores, fc.fc_marginals(ctx)


def _db(m, seed=3):
    return random_dag_database(12, m, 2, 5, 3, 0.7, seed=seed)


@pytest.mark.parametrize("cuts", [[1], [63, 64, 65], [4095, 1, 4097, 70_001], [100_000]])
def test_append_categorical_matches_single_load(cuts):
    torch = pytest.importorskip("torch")
    total = 1000 + sum(cuts)
    db = _db(total)
    D = np.ascontiguousarray(db.D)
    ctx = fc.fc_load(D[:, :1000], db.arities)
    gen0 = fc.fc_info(ctx, 5)
    p = 1000
    for i, c in enumerate(cuts):
        part = D[:, p:p + c]
        if i % 3 == 0:
            fc.fc_append(ctx, part)                                           # host, column-major
        elif i % 3 == 1:
            fc.fc_append(ctx, np.ascontiguousarray(part.T), fc.FC_ROW_MAJOR)  # host, row-major
        else:
            fc.fc_append(ctx, torch.from_numpy(np.ascontiguousarray(part)).cuda())  # device
        p += c
    assert fc.fc_info(ctx, 1) == total and fc.fc_info(ctx, 5) == gen0 + len(cuts)
    full = fc.fc_load(D, db.arities)
    queries = random_queries(db.n, 300, 1, 6, seed=5) + [[0, 1, 2, 3, 4, 5, 6, 7]]
    fams = [(q[-1], q[:-1]) for q in queries if len(q) <= 5]
    got = _all_results(ctx, queries, fams)
    want = _all_results(full, queries, fams)
    assert np.array_equal(got[0], want[0])
    for k in got[1]:
        assert np.array_equal(got[1][k], want[1][k]), k
    assert np.array_equal(got[2], want[2])
    # against the oracle on the concatenated database
    orc = oracle.DB(D, db.arities)
    off, _ = fc.pack_lists(queries)
    toff = np.concatenate([[0], np.cumsum([int(np.prod([db.arities[v] for v in q])) for q in queries])])
    for q in range(0, len(queries), 7):
        assert np.array_equal(got[0][toff[q]:toff[q + 1]].astype(np.int64), orc.table(queries[q]))
    for f in range(0, len(fams), 11):
        w = orc.score(fams[f][0], fams[f][1], "bdeu")
        assert abs(float(got[1]["bdeu"][f]) - w) <= 1e-5 * abs(w)
    marg = np.concatenate([np.bincount(D[v], minlength=int(db.arities[v])) for v in range(db.n)])
    assert np.array_equal(got[2], marg)


@pytest.mark.parametrize("arity", [(1, 2), (14, 16), (17, 40)])
def test_append_marginals_every_pack_path(arity):
    """Appended marginals come from the pack: bit planes (up to 16 states,
    arity-1 variables included) and two ballots per state (more states), at
    cuts inside and at the start of a bitmap word."""
    db = random_dag_database(7, 150_031, arity[0], arity[1], 2, 0.5, seed=17 + arity[1])
    D = np.ascontiguousarray(db.D)
    ctx = fc.fc_load(D[:, :40_001], db.arities)
    fc.fc_append(ctx, D[:, 40_001:40_064])          # up to a word boundary
    fc.fc_append(ctx, D[:, 40_064:150_031])
    marg = np.concatenate([np.bincount(D[v], minlength=int(db.arities[v])) for v in range(db.n)])
    assert np.array_equal(fc.fc_marginals(ctx), marg)
    orc = oracle.DB(D, db.arities)
    for q in ([0], [1, 2], [3, 0, 6]):
        assert np.array_equal(fc.fc_count(ctx, q).astype(np.int64), orc.table(q)), q


def test_append_all_paths_after_growth():
    """Bitmap DFS, histogram, sort, pairs, assignments and rules on a context
    grown past its first allocation, against a single load."""
    db = _db(300_000, seed=8)
    D = np.ascontiguousarray(db.D)
    ctx = fc.fc_load(D[:, :50_001], db.arities)
    cap0 = fc.fc_info(ctx, 4)
    fc.fc_append(ctx, D[:, 50_001:200_000])
    fc.fc_append(ctx, D[:, 200_000:])
    assert fc.fc_info(ctx, 4) > cap0
    full = fc.fc_load(D, db.arities)
    queries = random_queries(db.n, 120, 2, 6, seed=9)
    off, flat = fc.pack_lists(queries)
    for strat in (fc.FC_STRAT_BITMAP, fc.FC_STRAT_HIST, fc.FC_STRAT_SORT):
        for c in (ctx, full):
            fc.fc_set_option(c, "strategy", strat)
        assert np.array_equal(fc.fc_count_batch(ctx, off, flat)[0], fc.fc_count_batch(full, off, flat)[0]), strat
    for c in (ctx, full):
        fc.fc_set_option(c, "strategy", -1)
    t1, mi1 = fc.fc_pairs_all(ctx)
    t2, mi2 = fc.fc_pairs_all(full)
    assert np.array_equal(t1, t2) and np.array_equal(mi1, mi2)
    vo, vv = fc.pack_lists([q for q in queries])
    _, ss = fc.pack_lists([[v % 2 for v in q] for q in queries])
    assert np.array_equal(fc.fc_count_assignment_batch(ctx, vo, vv, ss),
                          fc.fc_count_assignment_batch(full, vo, vv, ss))
    r1, r2 = fc.fc_mine_rules(ctx, 0.2, 0.3, 5), fc.fc_mine_rules(full, 0.2, 0.3, 5)
    for k in ("set_off", "items", "support", "rule_set", "antecedent", "confidence"):
        assert np.array_equal(r1[k], r2[k]), k


def test_append_reserve_and_stale_plans():
    torch = pytest.importorskip("torch")
    db = _db(20_000, seed=4)
    D = np.ascontiguousarray(db.D)
    ctx = fc.fc_load(D[:, :10_000], db.arities)
    fc.fc_reserve(ctx, 1_000_000)
    cap = fc.fc_info(ctx, 4)
    assert cap >= 1_000_000
    queries = [[0, 1], [2, 3, 4]]
    off, flat = fc.pack_lists(queries)
    plan = fc.fc_plan_count(ctx, off, flat)
    out = torch.empty(fc.fc_plan_size(plan, 0), dtype=torch.int32, device="cuda")
    fc.fc_plan_run(plan, out)
    fc.fc_append(ctx, D[:, 10_000:])
    assert fc.fc_info(ctx, 4) == cap                     # no reallocation within the reserve
    with pytest.raises(fc.FcError) as e:
        fc.fc_plan_run(plan, out)
    assert e.value.code == fc.FC_ERR_STATE
    plan2 = fc.fc_plan_count(ctx, off, flat)
    fc.fc_plan_run(plan2, out)
    torch.cuda.synchronize()
    orc = oracle.DB(D, db.arities)
    want = np.concatenate([orc.table(q) for q in queries])
    assert np.array_equal(out.cpu().numpy().astype(np.int64), want)
    # freeing the context first orphans its plans: they refuse to run and
    # can still be freed
    ctx.close()
    with pytest.raises(fc.FcError) as e2:
        fc.fc_plan_run(plan2, out)
    assert e2.value.code == fc.FC_ERR_STATE
    plan2.close()
    plan.close()


def test_append_bad_state_changes_nothing():
    db = _db(5000, seed=6)
    D = np.ascontiguousarray(db.D)
    ctx = fc.fc_load(D[:, :3000], db.arities)
    marg0 = fc.fc_marginals(ctx)
    bad = D[:, 3000:].copy()
    bad[4, 17] = db.arities[4]                           # a state outside the arity
    with pytest.raises(fc.FcError) as e:
        fc.fc_append(ctx, bad)
    assert e.value.code == fc.FC_ERR_RANGE
    assert fc.fc_info(ctx, 1) == 3000 and np.array_equal(fc.fc_marginals(ctx), marg0)
    # the bitmaps hold the old rows only (the failed append was rolled back)
    old = fc.fc_load(D[:, :3000], db.arities)
    q_off, q_flat = fc.pack_lists([[4, 0], [1, 2, 3], [4]])
    for c in (ctx, old):
        fc.fc_set_option(c, "strategy", fc.FC_STRAT_BITMAP)
    assert np.array_equal(fc.fc_count_batch(ctx, q_off, q_flat)[0], fc.fc_count_batch(old, q_off, q_flat)[0])
    vo, vv = fc.pack_lists([[4, 0], [2]])
    _, ss = fc.pack_lists([[1, 0], [2]])
    assert np.array_equal(fc.fc_count_assignment_batch(ctx, vo, vv, ss), fc.fc_count_assignment_batch(old, vo, vv, ss))
    fc.fc_set_option(ctx, "strategy", -1)
    fc.fc_append(ctx, D[:, 3000:])                       # the valid rows still go in cleanly
    full = fc.fc_load(D, db.arities)
    off, flat = fc.pack_lists([[4, 0], [4, 1, 2]])
    assert np.array_equal(fc.fc_count_batch(ctx, off, flat)[0], fc.fc_count_batch(full, off, flat)[0])
    fc.fc_append(ctx, D[:, :0])                          # m_new = 0 is a no-op
    assert fc.fc_info(ctx, 1) == 5000
    with pytest.raises(fc.FcError):
        fc.fc_append_bits(ctx, np.zeros((db.n, 1), dtype=np.uint64), 10)


@pytest.mark.parametrize("cuts", [[1, 63, 64, 65, 1000], [4097, 130_001]])
def test_append_transactions(cuts):
    torch = pytest.importorskip("torch")
    total = 777 + sum(cuts)
    bits = basket_transaction_bitmaps(30, total, 5, seed=len(cuts))
    X = miner.item_matrix_from_bits(bits, total)
    ctx = fc.fc_load_bits(miner_pack(X[:, :777]), 777)
    p = 777
    for i, c in enumerate(cuts):
        part = miner_pack(X[:, p:p + c])
        if c % 64:
            part[:, -1] |= np.uint64(0xFFFFFFFFFFFFFFFF) << np.uint64(c % 64)   # garbage past m_new
        if i % 2:
            fc.fc_append_bits(ctx, torch.from_numpy(part.view(np.int64)).cuda(), c)
        else:
            fc.fc_append_bits(ctx, part, c)
        p += c
    assert fc.fc_info(ctx, 1) == total
    full = fc.fc_load_bits(bits, total)
    assert np.array_equal(fc.fc_marginals(ctx), X.sum(axis=1))
    sets = [[0, 5], [1, 6, 11], [2, 7, 12, 17], [0, 1, 2, 3, 4, 5, 6, 7, 8, 9], [29], []]
    so, it = fc.pack_lists(sets)
    a = fc.fc_support_batch(ctx, so, it)
    b = fc.fc_support_batch(full, so, it)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    for q, s in enumerate(sets[:-1]):
        assert int(a[0][q]) == miner.itemset_support(X, s)
    r1, r2 = fc.fc_mine_rules(ctx, 0.15, 0.4, 5, True), fc.fc_mine_rules(full, 0.15, 0.4, 5, True)
    for k in ("set_off", "items", "support", "rule_set", "antecedent", "confidence"):
        assert np.array_equal(r1[k], r2[k]), k


def miner_pack(X):
    m = X.shape[1]
    words = (m + 63) // 64
    pad = np.zeros((X.shape[0], words * 64), dtype=bool)
    pad[:, :m] = X
    return np.packbits(pad, axis=1, bitorder="little").view(np.uint64).reshape(X.shape[0], words).copy()
