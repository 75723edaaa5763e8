"""Seeded random configurations of the count planner against the oracle.

Each case draws a database (instances, arities including 1 and above 16),
a batch of queries (0 to 8 variables, repeated lists, tables from one cell to
beyond shared memory) and planner options (forced strategies, launch shapes,
window sizes, row-split sizes), then checks every table bit for bit.  The
cases cover combinations the targeted tests reach one at a time.
"""
import numpy as np
import pytest

import oracle
import paper_1804_04640_gb300 as fc
from workloads import random_dag_database, zipf_transaction_bitmaps

pytestmark = pytest.mark.gpu

OPTION_CHOICES = {
    "strategy": [fc.FC_STRAT_AUTO] * 4 + [fc.FC_STRAT_BITMAP, fc.FC_STRAT_HIST, fc.FC_STRAT_GATOMIC,
                                          fc.FC_STRAT_WINDOW],
    "min_part_rows": [4096, 8192, 65536],
    "window_cells": [1 << 20, 3001, 20000],
    "window_wide": [1, 1, 0],
    "window_max": [16, 4, 200],
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fc.load_library(build_if_missing=True)


@pytest.mark.parametrize("case", range(64))
def test_random_planner_configurations(case):
    rng = np.random.default_rng(9000 + case)
    n = int(rng.integers(2, 11))
    m = int(rng.choice([1, 63, 4097, 30_011, 130_003]))
    lo = int(rng.choice([1, 2, 3, 12]))
    hi = int(rng.choice([lo, lo + 2, 16, 40]))
    db = random_dag_database(n, m, lo, max(lo, hi), 2, float(rng.choice([0.3, 1.0])), seed=case)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    for key, vals in OPTION_CHOICES.items():
        fc.fc_set_option(ctx, key, int(vals[int(rng.integers(0, len(vals)))]))
    if rng.random() < 0.3:   # an explicit launch shape
        fc.fc_set_option(ctx, "smem_cells", int(rng.choice([2048, 8192, 16384])))
    nq = int(rng.choice([1, 7, 300, 5000]))
    queries = []
    for _ in range(nq):
        k = int(rng.integers(0, min(n, 8) + 1))
        vs = [int(x) for x in rng.choice(n, size=k, replace=False)]
        if np.prod([db.arities[v] for v in vs], dtype=np.float64) > 4e6:
            vs = vs[:2]
        queries.append(vs)
    off, flat = fc.pack_lists(queries)
    tables, toff = fc.fc_count_batch(ctx, off, flat)
    check = range(len(queries)) if len(queries) <= 300 else range(0, len(queries), 17)
    for q in check:
        want = orc.table(queries[q])
        got = tables[toff[q]:toff[q + 1]].astype(np.int64)
        assert np.array_equal(got, want), (case, q, queries[q])


@pytest.mark.parametrize("case", range(16))
def test_random_score_configurations(case):
    """Score plans under the same random options: every (child, parents)
    score within 1e-5 of the oracle's FP64 value (plus 1e-6 absolute for MI,
    whose value can be near zero)."""
    rng = np.random.default_rng(7000 + case)
    n = int(rng.integers(3, 12))
    m = int(rng.choice([17, 4097, 60_013, 200_003]))
    db = random_dag_database(n, m, int(rng.choice([1, 2])), int(rng.choice([3, 5, 9])), 3, 1.0, seed=50 + case)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    for key, vals in OPTION_CHOICES.items():
        fc.fc_set_option(ctx, key, int(vals[int(rng.integers(0, len(vals)))]))
    nq = int(rng.choice([1, 40, 5000]))
    child, parents = [], []
    for _ in range(nq):
        c = int(rng.integers(0, n))
        others = [v for v in range(n) if v != c]
        k = int(rng.integers(0, min(5, len(others)) + 1))
        child.append(c)
        parents.append([int(x) for x in rng.choice(others, size=k, replace=False)])
    po, pa = fc.pack_lists(parents)
    kind = ["ll", "mdl", "bdeu", "mi"][case % 4]
    got = fc.fc_score_batch(ctx, child, po, pa, kind, 1.0)
    check = range(nq) if nq <= 40 else range(0, nq, 53)
    for q in check:
        want = orc.score(child[q], parents[q], kind, 1.0)
        tol = 1e-5 * abs(want) + (1e-6 if kind == "mi" else 1e-12)
        assert abs(float(got[q]) - want) <= tol, (case, kind, q, child[q], parents[q], float(got[q]), want)


@pytest.mark.parametrize("case", range(16))
def test_random_support_configurations(case):
    """Itemset supports, leave-one-out supports, confidences and every
    antecedent split under random launch options, itemsets of 0 to 8 items
    (repeats allowed across itemsets)."""
    rng = np.random.default_rng(6000 + case)
    n_items = int(rng.integers(2, 81))
    m = int(rng.choice([1, 63, 64, 4097, 150_001]))
    bits = zipf_transaction_bitmaps(n_items, m, 1.1, float(rng.choice([2.0, 6.0])), seed=30 + case)
    ctx = fc.fc_load_bits(bits, m)
    fc.fc_set_option(ctx, "support_warps", int(rng.choice([1, 4, 16, 32])))
    fc.fc_set_option(ctx, "support_sets_per_warp", int(rng.choice([1, 4, 16])))
    fc.fc_set_option(ctx, "support_part_words", int(rng.choice([64, 512, 8192])))
    nq = int(rng.choice([1, 30, 2000]))
    sets = [[int(x) for x in rng.choice(n_items, size=int(rng.integers(0, min(8, n_items) + 1)), replace=False)]
            for _ in range(nq)]
    so, it = fc.pack_lists(sets)
    supp, sub, conf = fc.fc_support_batch(ctx, so, it)
    s2, sub2, conf2 = fc.fc_support_splits_batch(ctx, so, it)
    off = fc.split_offsets(so)
    check = range(nq) if nq <= 30 else range(0, nq, 41)
    for q in check:
        ws, wsub, wconf = oracle.support_rules(bits, m, sets[q])
        assert supp[q] == ws and s2[q] == ws, (case, q, sets[q])
        assert np.array_equal(sub[so[q]:so[q + 1]].astype(np.int64), wsub), (case, q)
        assert np.allclose(conf[so[q]:so[q + 1]], wconf, rtol=1e-6, atol=0), (case, q)
        ws2, wsub2, wconf2 = oracle.support_splits(bits, m, sets[q])
        assert np.array_equal(sub2[off[q]:off[q + 1]].astype(np.int64), wsub2), (case, q)
        assert np.allclose(conf2[off[q]:off[q + 1]], wconf2, rtol=1e-6, atol=0), (case, q)


@pytest.mark.parametrize("case", range(8))
def test_random_assignment_batches(case):
    """Specific assignments (end of Sec. 3.3): 0 to 6 conditions, states past
    the arity, a variable repeated with the same or another state."""
    rng = np.random.default_rng(5000 + case)
    n = int(rng.integers(2, 12))
    m = int(rng.choice([1, 65, 4097, 100_003]))
    db = random_dag_database(n, m, 1, int(rng.choice([3, 6, 20])), 2, 0.5, seed=70 + case)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    nq = int(rng.choice([1, 50, 3000]))
    vars_, states = [], []
    for _ in range(nq):
        k = int(rng.integers(0, 7))
        vs = [int(x) for x in rng.integers(0, n, size=k)]             # repeats allowed
        st = [int(rng.integers(0, db.arities[v] + (1 if rng.random() < 0.1 else 0))) for v in vs]
        vars_.append(vs)
        states.append(st)
    vo, vv = fc.pack_lists(vars_)
    _, ss = fc.pack_lists(states)
    got = fc.fc_count_assignment_batch(ctx, vo, vv, ss)
    check = range(nq) if nq <= 50 else range(0, nq, 29)
    for q in check:
        assert got[q] == orc.count_assignment(vars_[q], states[q]), (case, q, vars_[q], states[q])
