"""GPU parity of the bottom-up association-rule miner (Sec. 4.3).

fc_mine_rules must return exactly the oracle's frequent itemsets (same order,
same supports) and the same rules (itemset, antecedent mask); confidences are
the double quotient rounded once to float, compared with the oracle's double
within float rounding.
"""
import numpy as np
import pytest

import paper_1804_04640_gb300 as fc
from oracle import miner
from workloads import basket_transaction_bitmaps, config_database, random_dag_database

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    fc.load_library(build_if_missing=True)


def _compare(got, X, args):
    sets, supp, rules = miner.mine_rules(X, *args)
    so, it = got["set_off"], got["items"]
    gsets = [tuple(int(x) for x in it[so[i]:so[i + 1]]) for i in range(len(so) - 1)]
    assert gsets == sets, args
    assert got["support"].tolist() == supp, args
    assert list(zip(got["rule_set"].tolist(), got["antecedent"].tolist())) == [(i, mk) for i, mk, _ in rules]
    want = np.array([c for _, _, c in rules], dtype=np.float64)
    assert np.allclose(got["confidence"].astype(np.float64), want, rtol=2 ** -23, atol=0), args
    return len(sets), len(rules)


def _pack(X):
    m = X.shape[1]
    words = (m + 63) // 64
    pad = np.zeros((X.shape[0], words * 64), dtype=bool)
    pad[:, :m] = X
    return np.packbits(pad, axis=1, bitorder="little").view(np.uint64).reshape(X.shape[0], words)


def test_rules_hand_worked_transactions():
    txs = [[0, 1, 2], [0, 1], [0, 2], [0, 1, 2, 3], [1, 2], [3]]
    X = np.zeros((4, 6), dtype=bool)
    for p, t in enumerate(txs):
        X[t, p] = True
    ctx = fc.fc_load_bits(_pack(X), 6)
    for args in [(0.3, 0.6, 6, False), (0.3, 0.6, 6, True), (0.3, 0.4, 6, True), (0.5, 0.3, 6, False),
                 (0.3, 0.6, 2, False)]:
        _compare(fc.fc_mine_rules(ctx, *args), X, args)


@pytest.mark.parametrize("m", [1, 64, 4097, 70_001])
def test_rules_basket_transactions(m):
    bits = basket_transaction_bitmaps(24, m, 4, seed=m % 97 + 3)
    X = miner.item_matrix_from_bits(bits, m)
    ctx = fc.fc_load_bits(bits, m)
    total = 0
    for args in [(0.2, 0.3, 6, False), (0.1, 0.5, 5, True), (0.0, 0.0, 3, False), (0.35, 0.9, 32, False),
                 (0.2, 0.3, 1, True)]:
        ns, nr = _compare(fc.fc_mine_rules(ctx, *args), X, args)
        total += ns
    assert total > 0


def test_rules_categorical_items():
    """Items of a categorical database are (variable, state) events; two
    states of one variable never share an itemset."""
    db = random_dag_database(14, 30_011, 2, 4, 3, 1.0, seed=21)
    X = miner.item_matrix_from_db(db.D, db.arities)
    ctx = fc.fc_load(db.D, db.arities)
    for args in [(0.2, 0.3, 6, False), (0.1, 0.6, 4, True), (0.0, 0.0, 2, False)]:
        ns, nr = _compare(fc.fc_mine_rules(ctx, *args), X, args)
        assert ns > 0


def test_rules_levels_and_candidates():
    """Candidates counted on the device: every frequent set of size >= 2 was a
    candidate, and the search stops at the first empty level."""
    bits = basket_transaction_bitmaps(24, 20_000, 4, seed=1)
    ctx = fc.fc_load_bits(bits, 20_000)
    r = fc.fc_mine_rules(ctx, 0.2, 0.3, 32)
    sizes = np.diff(r["set_off"])
    assert r["candidates"] >= int((sizes >= 2).sum())
    assert int(sizes.max()) - 1 <= r["levels"] <= int(sizes.max())
    none = fc.fc_mine_rules(ctx, 1.0, 0.0, 6)
    assert len(none["support"]) == 0 and len(none["rule_set"]) == 0 and none["levels"] == 0


def test_rules_bad_arguments():
    bits = basket_transaction_bitmaps(8, 1000, 2, seed=2)
    ctx = fc.fc_load_bits(bits, 1000)
    for args in [(-0.1, 0.3, 6, False), (1.5, 0.3, 6, False), (0.2, -1.0, 6, False), (0.2, 0.3, 0, False),
                 (0.2, 0.3, 33, False), (0.2, 0.3, 17, True), (float("nan"), 0.3, 6, False)]:
        with pytest.raises(fc.FcError):
            fc.fc_mine_rules(ctx, *args)


def test_rules_bench_database_sampled():
    """The rules workload's database at a reduced row count, exact against the
    oracle (the full-size run is checked by properties in the bench-config
    tests)."""
    db = config_database("scores", 50_000)
    X = miner.item_matrix_from_db(db.D, db.arities)
    ctx = fc.fc_load(db.D, db.arities)
    ns, nr = _compare(fc.fc_mine_rules(ctx, 0.2, 0.3, 6), X, (0.2, 0.3, 6, False))
    assert ns > 1000 and nr > 1000
