"""GPU parity of the score reductions (Sec. 3.1): FP32 scores (BDeu as an LL
term plus FP32 remainders, FP64 only for per-query constants) within 1e-5
relative of the FP64 oracle, counts exact."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
import paper_1804_04640_gb300 as fc
from workloads import CONFIGS, config_database, random_dag_database, score_queries

pytestmark = pytest.mark.gpu
REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fc.load_library(build_if_missing=True)


def oracle_scores(orc, child, parents, kind, ess, idx):
    def one(q):
        return orc.score(child[q], parents[q], kind, ess)
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return np.array(list(ex.map(one, idx)))


def assert_close(got, want, what):
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - want)
    bad = err > REL * np.abs(want) + 1e-12
    assert not bad.any(), f"{what}: {int(bad.sum())} scores off, worst rel " \
        f"{float(np.max(err / np.maximum(np.abs(want), 1e-30)))}"


@pytest.mark.parametrize("kind", ["ll", "mdl", "bdeu", "mi"])
@pytest.mark.parametrize("strategy", [fc.FC_STRAT_AUTO, fc.FC_STRAT_BITMAP, fc.FC_STRAT_HIST,
                                      fc.FC_STRAT_GATOMIC, fc.FC_STRAT_SORT, fc.FC_STRAT_WINDOW])
def test_scores_small_all_queries(kind, strategy):
    db = random_dag_database(16, 90_001, 2, 4, 4, 1.0, seed=31)
    ctx = fc.fc_load(db.D, db.arities)
    fc.fc_set_option(ctx, "strategy", strategy)
    orc = oracle.DB(db.D, db.arities)
    child, parents = score_queries(db.n, 400, 0, 4, seed=32)
    po, pa = fc.pack_lists(parents)
    got = fc.fc_score_batch(ctx, child, po, pa, kind, 1.0)
    want = oracle_scores(orc, child, parents, kind, 1.0, range(len(child)))
    assert_close(got, want, kind)


@pytest.mark.parametrize("ess", [0.5, 4.0])
def test_bdeu_ess_and_row_splits(ess):
    """Few queries: rows are split across CTAs and the last CTA scores."""
    db = random_dag_database(10, 700_003, 2, 4, 3, 1.0, seed=41)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    child, parents = [0, 3, 5, 9], [[1, 2], [], [4, 6, 7, 8], [0]]
    po, pa = fc.pack_lists(parents)
    for kind in ("bdeu", "mdl", "mi"):
        got = fc.fc_score_batch(ctx, child, po, pa, kind, ess)
        want = oracle_scores(orc, child, parents, kind, ess, range(4))
        assert_close(got, want, kind)


@pytest.mark.parametrize("m", [1, 7, 8, 9, 1000, 1_000_003])
def test_bdeu_adversarial_tables(m):
    """Tables where the BDeu remainder terms matter most: deterministic and
    near-deterministic children (the LL part is ~0), counts at the switch
    between the small-count and Stirling branches, priors from 1e-3 to 100
    (a >= 1 takes the FP64 branch)."""
    rng = np.random.default_rng(m)
    n = 8
    D = np.zeros((n, m), dtype=np.uint8)
    D[0] = rng.integers(0, 4, size=m)                  # parent
    D[1] = D[0] % 2                                     # deterministic child of 0
    D[2] = np.where(rng.random(m) < 0.999, D[0] % 3, 2 - D[0] % 3)  # near-deterministic
    D[3] = 0                                            # constant
    D[4] = rng.integers(0, 2, size=m)
    D[5] = (D[4] + D[0]) % 2                            # deterministic given {0, 4}
    D[6] = rng.integers(0, 3, size=m)
    D[7] = rng.integers(0, 4, size=m)
    ar = [4, 2, 3, 1, 2, 2, 3, 4]
    ctx = fc.fc_load(D, ar)
    orc = oracle.DB(D, ar)
    child = [1, 2, 3, 5, 5, 1, 6, 7, 0]
    parents = [[0], [0], [0], [0, 4], [0, 4, 6, 7], [], [0, 1, 2, 4, 5], [6], [1, 2, 4, 5, 6, 7]]
    po, pa = fc.pack_lists(parents)
    for ess in (1e-3, 1.0, 10.0, 100.0):
        got = fc.fc_score_batch(ctx, child, po, pa, "bdeu", ess)
        want = oracle_scores(orc, child, parents, "bdeu", ess, range(len(child)))
        assert_close(got, want, f"bdeu ess={ess}")


def test_bn_score_workload_full_size_sampled():
    """Full BN-score workload (n=64, m=1e6, 50,000 queries): every score is
    computed on the GPU; a seeded sample of 1,500 is checked against the
    oracle, for MDL and BDeu (ESS = 1)."""
    c = CONFIGS["scores"]
    db = config_database("scores")
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    child, parents = score_queries(db.n, c["nq"], c["pa"][0], c["pa"][1], c["seed"])
    po, pa = fc.pack_lists(parents)
    idx = np.random.default_rng(7).choice(len(child), size=1500, replace=False)
    for kind in ("mdl", "bdeu"):
        got = fc.fc_score_batch(ctx, child, po, pa, kind, c["ess"])
        assert np.all(np.isfinite(got))
        want = oracle_scores(orc, child, parents, kind, c["ess"], idx)
        assert_close(got[idx], want, kind)


def test_score_plan_matches_host_call():
    torch = pytest.importorskip("torch")
    db = random_dag_database(20, 120_000, 2, 4, 3, 1.0, seed=51)
    ctx = fc.fc_load(db.D, db.arities)
    child, parents = score_queries(db.n, 3000, 0, 4, seed=52)
    po, pa = fc.pack_lists(parents)
    host = fc.fc_score_batch(ctx, child, po, pa, "bdeu", 1.0)
    plan = fc.fc_plan_score(ctx, child, po, pa, "bdeu", 1.0)
    out = torch.zeros(len(child), dtype=torch.float32, device="cuda")
    cur = torch.cuda.current_stream()
    for _ in range(2):
        fc.fc_plan_run(plan, out, stream=cur)
        fc.fc_sync(ctx, cur)
        assert np.array_equal(out.cpu().numpy(), host)


@pytest.mark.parametrize("kind", ["mdl", "bdeu", "mi", "ll"])
def test_family_lattice_scores(kind):
    """Every (child, parent set) family of a variable list (Sec. 4.2 query
    stream), each joint table counted once: against the oracle."""
    db = random_dag_database(14, 40_003, 2, 4, 3, 1.0, seed=81)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    vars_ = [3, 0, 11, 7, 5, 9, 12, 1, 4]
    fams = fc.family_list(vars_, 3)
    assert len(fams) == fc.fc_families_count(len(vars_), 3)
    got = fc.fc_score_families(ctx, vars_, 3, kind, 1.0)
    want = oracle_scores(orc, [f[0] for f in fams], [f[1] for f in fams], kind, 1.0, range(len(fams)))
    assert_close(got, want, kind)
    # the same families through the per-query score batch
    po, pa = fc.pack_lists([f[1] for f in fams])
    direct = fc.fc_score_batch(ctx, [f[0] for f in fams], po, pa, kind, 1.0)
    assert_close(direct, want, kind)
