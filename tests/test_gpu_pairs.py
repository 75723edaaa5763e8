"""GPU parity of the all-pairs one-hot co-occurrence product (tcgen05) and of
the mutual information of every pair."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
import paper_1804_04640_gb300 as fc
from workloads import config_database, random_dag_database

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fc.load_library(build_if_missing=True)


def pair_index(n):
    return [(a, b) for a in range(n) for b in range(a + 1, n)]


def pair_offsets(ar):
    n = len(ar)
    off = [0]
    for a, b in pair_index(n):
        off.append(off[-1] + int(ar[a]) * int(ar[b]))
    return np.array(off, dtype=np.int64)


def check_pairs(db, idx):
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    tables, mi = fc.fc_pairs_all(ctx)
    pairs = pair_index(db.n)
    off = pair_offsets(db.arities)
    marg = fc.fc_marginals(ctx)
    soff = np.concatenate([[0], np.cumsum(db.arities)])
    # properties that hold for every pair at any size
    for p, (a, b) in enumerate(pairs):
        t = tables[off[p]:off[p + 1]].reshape(int(db.arities[a]), int(db.arities[b])).astype(np.int64)
        assert t.sum() == db.m
        assert np.array_equal(t.sum(axis=1), marg[soff[a]:soff[a + 1]])
        assert np.array_equal(t.sum(axis=0), marg[soff[b]:soff[b + 1]])
    assert np.all(mi[: len(pairs)] >= 0)

    def one(p):
        a, b = pairs[p]
        t = orc.table([a, b])
        return t, oracle.score_table(t, int(db.arities[a]), int(db.arities[b]), "mi")

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        res = list(ex.map(one, idx))
    for p, (t, want_mi) in zip(idx, res):
        assert np.array_equal(tables[off[p]:off[p + 1]].astype(np.int64), t), pairs[p]
        assert abs(float(mi[p]) - want_mi) <= 1e-5 * abs(want_mi) + 1e-12, (pairs[p], mi[p], want_mi)
    return ctx


@pytest.mark.parametrize("n,m,seed", [(20, 5_000, 1), (7, 131, 2), (40, 100_003, 3), (90, 64, 4)])
def test_pairs_small_all(n, m, seed):
    db = random_dag_database(n, m, 2, 5, 2, 0.5, seed=seed)
    check_pairs(db, list(range(n * (n - 1) // 2)))


def test_pairs_high_arity_spans_many_tiles():
    db = random_dag_database(30, 20_001, 8, 20, 2, 0.5, seed=5)   # sum of arities > 256
    check_pairs(db, list(range(30 * 29 // 2)))


def test_pairs_full_workload_sampled():
    """All-pairs workload (n=256, m=1e6): every pair checked by its
    invariants, 400 seeded pairs against the oracle's row scan."""
    db = config_database("pairs")
    npairs = db.n * (db.n - 1) // 2
    idx = sorted(np.random.default_rng(3).choice(npairs, size=400, replace=False).tolist())
    check_pairs(db, idx)


def test_pairs_plan_replay_and_chunked_accumulation():
    torch = pytest.importorskip("torch")
    db = random_dag_database(50, 300_000, 2, 3, 2, 0.5, seed=6)
    ctx = fc.fc_load(db.D, db.arities)
    t0, m0 = fc.fc_pairs_all(ctx)
    fc.fc_set_option(ctx, "pair_chunk_rows", 4096)        # many short row splits
    t1, m1 = fc.fc_pairs_all(ctx)
    assert np.array_equal(t0, t1)
    assert np.allclose(m0, m1, rtol=1e-6, atol=0)
    plan = fc.fc_plan_pairs(ctx)
    out_t = torch.zeros(fc.fc_plan_size(plan, 0), dtype=torch.int32, device="cuda")
    out_m = torch.zeros(fc.fc_plan_size(plan, 1), dtype=torch.float32, device="cuda")
    cur = torch.cuda.current_stream()
    for _ in range(2):
        fc.fc_plan_run(plan, out_t, out_m, stream=cur)
        fc.fc_sync(ctx, cur)
        assert np.array_equal(out_t.cpu().numpy(), t1)


def test_pairs_into_page_locked_outputs():
    """fc_pairs_all into page-locked buffers: the extraction kernel stores the
    tables and the MI straight into them (option zero_copy); the results
    equal the copied ones, for both outputs, either one alone, and with the
    option off."""
    torch = pytest.importorskip("torch")
    db = random_dag_database(40, 100_003, 2, 4, 2, 0.5, seed=9)
    ctx = fc.fc_load(db.D, db.arities)
    t0, m0 = fc.fc_pairs_all(ctx)
    lib = fc.load_library()
    for zc in (1, 0):
        fc.fc_set_option(ctx, "zero_copy", zc)
        for want_t, want_m in ((True, True), (True, False), (False, True)):
            pt = torch.full((len(t0),), -7, dtype=torch.int32).pin_memory() if want_t else None
            pm = torch.full((len(m0),), -7.0, dtype=torch.float32).pin_memory() if want_m else None
            rc = lib.fc_pairs_all(ctx.ptr, fc._ptr(pt), fc._ptr(pm))
            assert rc == fc.FC_OK, fc.fc_last_error()
            if want_t:
                assert np.array_equal(pt.numpy(), t0)
            if want_m:
                assert np.array_equal(pm.numpy(), m0)
    fc.fc_set_option(ctx, "zero_copy", 1)
