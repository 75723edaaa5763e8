"""Pins of the CPU oracle to facts other than itself (CPU only).

Each test ties one oracle function to something the paper or mathematics
fixes independently: the worked example of Sec. 2, brute-force enumeration of
assignments on tiny databases, table invariants (sums, marginals, axis
permutation, N_ij = sum_k N_ijk from Eq. 1), closed forms of the scores on
special tables, library routines (scipy entropy, scikit-learn mutual
information), a gamma-free sequential form of the Dirichlet marginal
likelihood, and brute-force support counts over transaction lists.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from workloads import random_dag_database, zipf_transaction_bitmaps

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows, kv = [], {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if parts[0].isalpha():
            kv[parts[0]] = parts[1:]
        else:
            rows.append([int(x) for x in parts])
    return rows, kv


def test_worked_example_count():
    """Sec. 2: Count((X1=3) and (X2=2) and (X3=1)) = 2."""
    rows, kv = _read_golden("worked_example.txt")
    ar = [int(x) for x in kv["arities"]]
    D1 = np.array(rows, dtype=np.int64).T          # (n, m), 1-based states
    db = oracle.DB((D1 - 1).astype(np.uint8), ar)  # stored 0-based
    q = [int(x) for x in kv["query"]]
    vars_ = [q[0] - 1, q[2] - 1, q[4] - 1]
    states = [q[1] - 1, q[3] - 1, q[5] - 1]
    assert db.count_assignment(vars_, states) == int(kv["expect"][0])
    # the same count is the matching cell of the full table
    t = db.table(vars_)
    idx = np.ravel_multi_index(tuple(states), tuple(ar[v] for v in vars_))
    assert t[idx] == 2


def _tiny_dbs():
    out = []
    for seed, (n, m) in enumerate([(3, 1), (3, 17), (4, 64), (4, 33), (2, 64)]):
        out.append(random_dag_database(n, m, 1 if seed == 0 else 2, 4, 2, 0.7, 100 + seed))
    return out


@pytest.mark.parametrize("db", _tiny_dbs(), ids=lambda d: f"n{d.n}m{d.m}")
def test_table_brute_force_all_subsets(db):
    """Every ordered variable list of a tiny database: each cell equals an
    independent count of the rows that match that assignment, enumerated in
    lexicographic order (last variable fastest)."""
    o = oracle.DB(db.D, db.arities)
    for k in range(0, db.n + 1):
        for vars_ in itertools.permutations(range(db.n), k):
            t = o.table(list(vars_))
            shape = [int(db.arities[v]) for v in vars_]
            expect = []
            for assign in itertools.product(*[range(s) for s in shape]):
                c = 0
                for p in range(db.m):
                    if all(int(db.D[v, p]) == s for v, s in zip(vars_, assign)):
                        c += 1
                expect.append(c)
            assert t.tolist() == expect, (vars_,)


def test_table_invariants():
    db = random_dag_database(10, 5000, 2, 5, 3, 0.5, 7)
    o = oracle.DB(db.D, db.arities)
    rng = np.random.default_rng(0)
    for _ in range(30):
        k = int(rng.integers(1, 5))
        vars_ = [int(x) for x in rng.choice(db.n, size=k, replace=False)]
        shape = [int(db.arities[v]) for v in vars_]
        t = o.table(vars_).reshape(shape)
        assert t.sum() == db.m                              # tables sum to m
        for ax in range(k):                                 # marginal = lower-order table
            sub = vars_[:ax] + vars_[ax + 1:]
            assert np.array_equal(t.sum(axis=ax).reshape(-1), o.table(sub))
        perm = list(rng.permutation(k))                     # permuting vars permutes axes
        tp = o.table([vars_[i] for i in perm]).reshape([shape[i] for i in perm])
        assert np.array_equal(tp, np.transpose(t, perm))
        # single-variable tables are histograms of the column (library routine)
        assert np.array_equal(o.table([vars_[0]]),
                              np.bincount(db.D[vars_[0]], minlength=shape[0]))


def test_table_rejects_bad_input():
    db = random_dag_database(4, 50, 2, 3, 1, 1.0, 3)
    o = oracle.DB(db.D, db.arities)
    with pytest.raises(oracle.OracleError):
        o.table([0, 0])
    bad = oracle.DB(np.full((2, 5), 3, dtype=np.uint8), [3, 3])
    with pytest.raises(oracle.OracleError):
        bad.table([0])
    assert o.table([]).tolist() == [db.m]                   # k = 0: one cell = m


def test_hand_worked_scores():
    _, kv = _read_golden("hand_scores.txt")
    t = np.array([int(x) for x in kv["table"]], dtype=np.int64)
    q, r = int(kv["q"][0]), int(kv["r"][0])
    for kind in ("ll", "mdl", "mi"):
        assert oracle.score_table(t, q, r, kind) == pytest.approx(float(kv[kind][0]), abs=1e-12)


def test_ll_closed_forms():
    scipy_stats = pytest.importorskip("scipy.stats")
    db = random_dag_database(6, 20000, 2, 5, 2, 0.5, 11)
    o = oracle.DB(db.D, db.arities)
    for x in range(db.n):
        # empty parent set: LL = -m H(X) in bits
        cnt = np.bincount(db.D[x], minlength=int(db.arities[x]))
        h = scipy_stats.entropy(cnt, base=2)
        assert o.score(x, [], "ll") == pytest.approx(-db.m * h, rel=1e-12)
    # deterministic child (a copy of its parent): LL = 0
    D2 = np.vstack([db.D[0], db.D[0]])
    o2 = oracle.DB(D2, [db.arities[0]] * 2)
    assert o2.score(1, [0], "ll") == 0.0
    # uniform 2x2 table: LL = -m
    t = np.array([5, 5, 5, 5], dtype=np.int64)
    assert oracle.score_table(t, 2, 2, "ll") == pytest.approx(-20.0, abs=1e-12)


def test_mdl_penalty_counts_all_parent_configurations():
    """The MDL penalty uses q = product of parent arities even when some
    configurations never occur: a deterministic child (LL = 0) scores the
    penalty alone, (log2 m / 2) (r - 1) q."""
    D = np.array([[0, 1, 0, 1, 0, 1, 0, 1], [0, 1, 0, 1, 0, 1, 0, 1]], dtype=np.uint8)
    o = oracle.DB(D, [3, 2])    # X0 has 3 states, state 2 never observed
    assert o.score(1, [0], "mdl") == pytest.approx(0.5 * 3 * 1 * 3, abs=1e-12)


def _polya_log_marginal(D, child, parents, arities, ess):
    """Dirichlet-multinomial marginal likelihood by the sequential predictive
    (Polya urn) rule: each row in turn has probability
    (n_jk + a_jk) / (n_j + a_j) given the rows before it.  No gamma function."""
    r = int(arities[child])
    q = int(np.prod([int(arities[p]) for p in parents])) if parents else 1
    a_j, a_jk = ess / q, ess / (r * q)
    nj, njk = {}, {}
    total = 0.0
    for p in range(D.shape[1]):
        j = tuple(int(D[v, p]) for v in parents)
        k = int(D[child, p])
        total += math.log((njk.get((j, k), 0) + a_jk) / (nj.get(j, 0) + a_j))
        nj[j] = nj.get(j, 0) + 1
        njk[(j, k)] = njk.get((j, k), 0) + 1
    return total


@pytest.mark.parametrize("ess", [1.0, 0.25, 10.0])
def test_bdeu_matches_polya_urn(ess):
    db = random_dag_database(5, 300, 2, 4, 2, 0.5, 21)
    o = oracle.DB(db.D, db.arities)
    for child, parents in [(0, []), (1, [0]), (2, [0, 1]), (4, [3, 2, 1]), (3, [4])]:
        expect = _polya_log_marginal(db.D, child, parents, db.arities, ess)
        assert o.score(child, parents, "bdeu", ess) == pytest.approx(expect, rel=1e-11, abs=1e-9)


def test_mi_closed_forms_and_library():
    scipy_stats = pytest.importorskip("scipy.stats")
    db = random_dag_database(6, 20000, 2, 5, 2, 0.5, 13)
    o = oracle.DB(db.D, db.arities)
    # MI(X; X) = H(X)
    D2 = np.vstack([db.D[2], db.D[2]])
    o2 = oracle.DB(D2, [db.arities[2]] * 2)
    h = scipy_stats.entropy(np.bincount(db.D[2]), base=2)
    assert o2.score(1, [0], "mi") == pytest.approx(h, rel=1e-12)
    # a product table has MI = 0
    a, b = np.array([3, 5, 2]), np.array([7, 1, 4, 4])
    assert abs(oracle.score_table(np.outer(a, b).reshape(-1), 3, 4, "mi")) < 1e-14
    # MI = H(X) + H(Y) - H(X, Y), and MI >= 0
    for x, y in [(0, 1), (2, 3), (4, 5), (1, 4)]:
        t = o.table([y, x])
        hx = scipy_stats.entropy(np.bincount(db.D[x]), base=2)
        hy = scipy_stats.entropy(np.bincount(db.D[y]), base=2)
        hxy = scipy_stats.entropy(t[t > 0], base=2)
        mi = o.score(x, [y], "mi")
        assert mi == pytest.approx(hx + hy - hxy, rel=1e-10, abs=1e-12)
        assert mi >= 0.0
    # the joint parent configuration acts as one variable; check against
    # scikit-learn's mutual information (natural log) when available
    try:
        from sklearn.metrics import mutual_info_score
    except Exception:  # pragma: no cover - the GPU image has no scikit-learn
        return
    y_joint = db.D[0].astype(np.int64) * 10 + db.D[1]
    mi_nats = mutual_info_score(db.D[3], y_joint)
    assert o.score(3, [0, 1], "mi") == pytest.approx(mi_nats / math.log(2), rel=1e-9)


def test_support_rules_brute_force():
    m = 200
    bits = zipf_transaction_bitmaps(12, m, 1.1, 3.0, 31)
    # transaction lists from the bitmaps (numpy unpack, library routine)
    holds = np.unpackbits(bits.view(np.uint8), axis=1, bitorder="little")[:, :m].astype(bool)
    trans = [set(np.nonzero(holds[:, p])[0].tolist()) for p in range(m)]
    rng = np.random.default_rng(3)
    for _ in range(40):
        k = int(rng.integers(1, 6))
        items = sorted(int(x) for x in rng.choice(12, size=k, replace=False))
        supp, sub, conf = oracle.support_rules(bits, m, items)
        assert supp == sum(1 for T in trans if set(items) <= T)
        for t in range(k):
            rest = set(items) - {items[t]}
            s = sum(1 for T in trans if rest <= T)
            assert sub[t] == s and supp <= s             # anti-monotone
            assert conf[t] == (supp / s if s else 0.0)
            assert 0.0 <= conf[t] <= 1.0
    # supp(empty set) = m, supp({i}) = popcount of bitmap i
    assert oracle.support_rules(bits, m, [])[0] == m
    for i in range(12):
        assert oracle.support_rules(bits, m, [i])[0] == int(holds[i].sum())


def test_support_splits_brute_force():
    """Every antecedent split of an itemset against transaction lists; the
    single-consequent masks agree with the leave-one-out supports."""
    m = 150
    bits = zipf_transaction_bitmaps(10, m, 1.1, 4.0, 37)
    holds = np.unpackbits(bits.view(np.uint8), axis=1, bitorder="little")[:, :m].astype(bool)
    trans = [set(np.nonzero(holds[:, p])[0].tolist()) for p in range(m)]
    rng = np.random.default_rng(4)
    for _ in range(25):
        k = int(rng.integers(0, 6))
        items = [int(x) for x in rng.choice(10, size=k, replace=False)]
        supp, sub, conf = oracle.support_splits(bits, m, items)
        assert supp == sum(1 for T in trans if set(items) <= T)
        assert len(sub) == max((1 << k) - 2, 0)
        for mask in range(1, (1 << k) - 1):
            A = {items[t] for t in range(k) if mask >> t & 1}
            s = sum(1 for T in trans if A <= T)
            assert sub[mask - 1] == s and supp <= s
            assert conf[mask - 1] == (supp / s if s else 0.0)
        if k >= 2:
            s1, loo, _ = oracle.support_rules(bits, m, items)
            full = (1 << k) - 1
            assert [sub[(full ^ (1 << t)) - 1] for t in range(k)] == loo.tolist()


# ---- association-rule miner (Sec. 4.3) -------------------------------------

def _rules_cases():
    txs, cases, cur = [], [], None
    for line in open(os.path.join(GOLDEN, "rules_example.txt")):
        tok = line.split()
        if not tok or tok[0].startswith("#"):
            continue
        if tok[0] == "tx":
            txs.append([int(x) for x in tok[1:]])
        elif tok[0] == "case":
            cur = {"args": (float(tok[1]), float(tok[2]), int(tok[3]), bool(int(tok[4]))),
                   "sets": [], "rules": []}
        elif tok[0] == "set":
            i = tok.index(":")
            cur["sets"].append((tuple(int(x) for x in tok[1:i]), int(tok[i + 1])))
        elif tok[0] == "rule":
            a, b = tok[3].split("/")
            cur["rules"].append((int(tok[1]), int(tok[2]), int(a) / int(b)))
        elif tok[0] == "end":
            cases.append(cur)
    X = np.zeros((4, len(txs)), dtype=bool)
    for p, t in enumerate(txs):
        X[t, p] = True
    return X, cases


def test_rules_hand_worked():
    """Frequent itemsets and rules of a hand-worked six-transaction database,
    including the strict thresholds and the size limit."""
    from oracle import miner
    X, cases = _rules_cases()
    assert len(cases) == 5
    for c in cases:
        sets, supp, rules = miner.mine_rules(X, *c["args"])
        assert list(zip(sets, supp)) == c["sets"], c["args"]
        assert [(i, mk) for i, mk, _ in rules] == [(i, mk) for i, mk, _ in c["rules"]], c["args"]
        for (_, _, got), (_, _, want) in zip(rules, c["rules"]):
            assert got == pytest.approx(want, rel=1e-15)


def _brute_rules(X, min_support, min_confidence, max_size, all_splits):
    """Every subset of at most max_size items, counted with a row loop."""
    n, m = X.shape
    rows = [set(np.flatnonzero(X[:, p]).tolist()) for p in range(m)]

    def supp(S):
        return sum(1 for r in rows if all(i in r for i in S))

    sets = []
    for k in range(1, max_size + 1):
        for S in itertools.combinations(range(n), k):
            s = supp(S)
            if s > min_support * m:
                sets.append((S, s))
    rules = []
    for idx, (S, s) in enumerate(sets):
        k = len(S)
        for mask in range(1, (1 << k) - 1):
            if not all_splits and bin(mask).count("1") != k - 1:
                continue
            a = supp([S[t] for t in range(k) if mask >> t & 1])
            if s > min_confidence * a:
                rules.append((idx, mask, s / a))
    return sets, rules


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rules_brute_force(seed):
    """The level-wise search equals counting every subset of at most max_size
    items directly (correlated items so that sets of 4-5 items are frequent)."""
    from oracle import miner
    rng = np.random.default_rng(seed)
    n, m = 10, 120
    base = rng.random(m) < 0.7
    X = np.array([(base & (rng.random(m) < 0.9)) | (rng.random(m) < 0.2) for _ in range(n)])
    for args in [(0.25, 0.5, 5, False), (0.3, 0.7, 4, True), (0.05, 0.0, 3, True), (0.9, 0.3, 6, False)]:
        sets, supp, rules = miner.mine_rules(X, *args)
        bsets, brules = _brute_rules(X, *args)
        assert sorted(zip(sets, supp)) == sorted(bsets)
        # order: size by size, lexicographic within a size
        assert sets == sorted(sets, key=lambda S: (len(S), S))
        got = {(sets[i], mk): c for i, mk, c in rules}
        want = {(bsets[i][0], mk): c for i, mk, c in brules}
        assert got.keys() == want.keys() and all(got[k] == pytest.approx(want[k], rel=1e-15) for k in got)
    assert max(len(S) for S in miner.mine_rules(X, 0.25, 0.5, 6)[0]) >= 4


def test_rules_item_matrices():
    """Item ids of a categorical database are (variable, state) pairs in
    arity order; bitmaps unpack least significant bit first."""
    from oracle import miner
    D = np.array([[0, 1, 2, 1], [1, 1, 0, 0]], dtype=np.uint8)
    X = miner.item_matrix_from_db(D, [3, 2])
    assert X.shape == (5, 4)
    assert X[2].tolist() == [False, False, True, False] and X[3].tolist() == [False, False, True, True]
    bits = np.array([[0b1011], [1 << 63 | 1]], dtype=np.uint64)
    Y = miner.item_matrix_from_bits(bits, 64)
    assert Y[0, :4].tolist() == [True, True, False, True] and Y[0].sum() == 3
    assert Y[1, 0] and Y[1, 63] and Y[1].sum() == 2
    assert miner.itemset_support(X, []) == 4 and miner.itemset_support(X, [1, 3]) == 1
