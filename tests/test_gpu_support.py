"""GPU parity of itemset support and rule confidence (Sec. 4.3)."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
import paper_1804_04640_gb300 as fc
from workloads import CONFIGS, weighted_itemsets, zipf_item_probs, zipf_transaction_bitmaps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fc.load_library(build_if_missing=True)


def check(bits, m, sets, idx, got):
    supp, sub, conf = got
    so, _ = fc.pack_lists(sets)

    def one(q):
        return oracle.support_rules(bits, m, sets[q])

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        res = list(ex.map(one, idx))
    for q, (s, sb, cf_) in zip(idx, res):
        a, b = so[q], so[q + 1]
        assert supp[q] == s, (q, sets[q])
        assert np.array_equal(sub[a:b].astype(np.int64), sb), (q, sets[q])
        assert np.allclose(conf[a:b], cf_, rtol=1e-6, atol=0), (q, conf[a:b], cf_)


@pytest.mark.parametrize("m", [1, 63, 64, 65, 4097, 200_003])
def test_support_small_all(m):
    bits = zipf_transaction_bitmaps(40, m, 1.1, 6.0, seed=m % 1000 + 1)
    probs = zipf_item_probs(40, 1.1, 6.0)
    sets = weighted_itemsets(40, 500, 2, 9, probs, seed=2) + [[3], [7], [], [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10]]
    ctx = fc.fc_load_bits(bits, m)
    so, it = fc.pack_lists(sets)
    got = fc.fc_support_batch(ctx, so, it)
    check(bits, m, sets, list(range(len(sets))), got)


def test_support_split_words():
    """Many word ranges per itemset: partial supports summed atomically."""
    m = 1_000_003
    bits = zipf_transaction_bitmaps(30, m, 1.1, 5.0, seed=4)
    sets = weighted_itemsets(30, 300, 2, 5, zipf_item_probs(30, 1.1, 5.0), seed=5)
    ctx = fc.fc_load_bits(bits, m)
    fc.fc_set_option(ctx, "support_part_words", 64)
    so, it = fc.pack_lists(sets)
    check(bits, m, sets, list(range(len(sets))), fc.fc_support_batch(ctx, so, it))


def test_support_full_workload_sampled():
    """Association-rule workload: 1,000 items, m = 1e7, 1e6 itemsets of size
    2-5.  All supports are computed on the GPU; 48 seeded itemsets are
    checked against the oracle's transaction scan and every itemset against
    properties that hold at any size."""
    c = CONFIGS["support"]
    m = c["m"]
    bits = zipf_transaction_bitmaps(c["n_items"], m, c["zipf_s"], c["mean_len"], c["seed"])
    probs = zipf_item_probs(c["n_items"], c["zipf_s"], c["mean_len"])
    sets = weighted_itemsets(c["n_items"], c["nq"], c["k"][0], c["k"][1], probs, c["seed"])
    ctx = fc.fc_load_bits(bits, m)
    so, it = fc.pack_lists(sets)
    supp, sub, conf = fc.fc_support_batch(ctx, so, it)
    item_supp = fc.fc_marginals(ctx)
    k = np.diff(so)
    # anti-monotone, confidence in [0, 1] and equal to supp / sub
    owner = np.repeat(np.arange(len(sets)), k)
    assert np.all(supp[owner] <= sub)
    assert np.all((conf >= 0) & (conf <= 1))
    ratio = np.where(sub > 0, supp[owner] / np.maximum(sub, 1), 0.0)
    assert np.allclose(conf, ratio, rtol=1e-6, atol=0)
    # for pairs, the leave-one-out supports are the single-item supports
    two = np.nonzero(k == 2)[0]
    a = so[two]
    assert np.array_equal(sub[a], item_supp[it[a + 1]])
    assert np.array_equal(sub[a + 1], item_supp[it[a]])
    idx = sorted(np.random.default_rng(11).choice(len(sets), size=48, replace=False).tolist())
    check(bits, m, sets, idx, (supp, sub, conf))


def check_splits(bits, m, sets, idx, got):
    supp, sub, conf = got
    so, _ = fc.pack_lists(sets)
    off = fc.split_offsets(so)

    def one(q):
        return oracle.support_splits(bits, m, sets[q])

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        res = list(ex.map(one, idx))
    for q, (s, sb, cf_) in zip(idx, res):
        a, b = off[q], off[q + 1]
        assert supp[q] == s, (q, sets[q])
        assert np.array_equal(sub[a:b].astype(np.int64), sb), (q, sets[q])
        assert np.allclose(conf[a:b], cf_, rtol=1e-6, atol=0), (q, conf[a:b], cf_)


@pytest.mark.parametrize("m", [1, 64, 65, 4097, 200_003])
def test_support_splits_all(m):
    """Every antecedent split (2^k - 2 per itemset), sizes 0 to 9 (the
    unrolled walk covers 2-6, the generic loop the rest)."""
    bits = zipf_transaction_bitmaps(40, m, 1.1, 6.0, seed=m % 997 + 5)
    probs = zipf_item_probs(40, 1.1, 6.0)
    sets = weighted_itemsets(40, 300, 2, 7, probs, seed=3) + [[3], [], [0, 1, 2, 3, 4, 5, 6, 7, 8]]
    ctx = fc.fc_load_bits(bits, m)
    so, it = fc.pack_lists(sets)
    got = fc.fc_support_splits_batch(ctx, so, it)
    check_splits(bits, m, sets, range(len(sets)), got)
    # the single-consequent masks equal the leave-one-out supports
    s1, sub1, _ = fc.fc_support_batch(ctx, so, it)
    off = fc.split_offsets(so)
    for q, S in enumerate(sets):
        k = len(S)
        if k >= 2:
            full = (1 << k) - 1
            want = sub1[so[q]:so[q + 1]]
            got_loo = [got[1][off[q] + (full ^ (1 << t)) - 1] for t in range(k)]
            assert np.array_equal(np.array(got_loo), want)
    assert np.array_equal(got[0][:len(sets)], s1[:len(sets)])


def test_support_splits_row_ranges_and_plan():
    """Long bitmaps split into word ranges (atomic partial counts), through a
    device-resident plan replayed twice."""
    torch = pytest.importorskip("torch")
    m = 1_000_003
    bits = zipf_transaction_bitmaps(30, m, 1.1, 8.0, seed=77)
    probs = zipf_item_probs(30, 1.1, 8.0)
    sets = weighted_itemsets(30, 200, 2, 6, probs, seed=8)
    ctx = fc.fc_load_bits(bits, m)
    fc.fc_set_option(ctx, "support_part_words", 2048)
    so, it = fc.pack_lists(sets)
    plan = fc.fc_plan_support_splits(ctx, so, it)
    ns = fc.fc_plan_size(plan, 3)
    assert ns == int(fc.split_offsets(so)[-1])
    outs = [torch.empty(len(sets), dtype=torch.int32, device="cuda"),
            torch.empty(ns, dtype=torch.int32, device="cuda"),
            torch.empty(ns, dtype=torch.float32, device="cuda")]
    res = []
    for _ in range(2):
        fc.fc_plan_run(plan, *outs)
        torch.cuda.synchronize()
        res.append([o.cpu().numpy().copy() for o in outs])
    for a, b in zip(*res):
        assert np.array_equal(a, b)
    idx = np.random.default_rng(1).choice(len(sets), size=24, replace=False)
    check_splits(bits, m, sets, idx, res[1])
    with pytest.raises(fc.FcError):
        fc.fc_support_splits_batch(ctx, *fc.pack_lists([list(range(17))]))
