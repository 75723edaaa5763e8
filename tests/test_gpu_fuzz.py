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
from workloads import random_dag_database

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


@pytest.mark.parametrize("case", range(24))
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
