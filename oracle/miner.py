"""CPU oracle of the bottom-up association-rule miner (test infrastructure).

Only the test suite and the CPU-baseline leg of ``bench.py`` may import this
module; the library never touches it and the two share no code.

Sec. 4.3 of the paper mines rules ``Pa => X`` over binary items: an itemset S
is frequent when the fraction of transactions holding every item of S is above
a support threshold, and a rule A => S \\ A drawn from a frequent S is kept when
its confidence supp(S) / supp(A) is above a confidence threshold.  The search
goes bottom-up over the power-set lattice, one itemset size at a time, and
stops at a maximum itemset size.

Readings (the paper states the thresholds as strict inequalities):
  * frequent:  supp(S) > min_support * m, decided in double precision;
  * rule kept: supp(S) > min_confidence * supp(A), decided in double precision;
  * itemsets are lists of item ids in increasing order, listed size by size
    and lexicographically within a size;
  * a rule is (index of S, antecedent mask): bit t set when position t of S
    is in the antecedent A; the consequent is the rest of S.  With
    ``all_splits`` every non-empty proper subset of S is an antecedent
    (2^k - 2 rules per itemset); otherwise only single-item consequents
    (k rules per itemset), the form ``Pa(X_i) => X_i`` the paper names.

Items of a categorical database are the pairs (variable v, state s), item id
``sum(arities[:v]) + s``: a transaction holds the item when D[v, p] == s.

The steps follow the plain level-wise search: level 1 counts every item;
level k extends each frequent (k-1)-set S by every larger item j for which
all k of the (k-1)-subsets of S + (j,) are frequent (a set with an infrequent
subset cannot be frequent, since support only falls as items are added), then
counts each such candidate directly by scanning the item matrix.
"""
from __future__ import annotations

import numpy as np


def item_matrix_from_bits(bits: np.ndarray, m: int) -> np.ndarray:
    """(n_items, m) bool matrix of 64-bit little-endian transaction bitmaps."""
    b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint64))
    as_bytes = b.view(np.uint8).reshape(b.shape[0], -1)
    X = np.unpackbits(as_bytes, axis=1, bitorder="little")[:, :m]
    return X.astype(bool)


def item_matrix_from_db(D: np.ndarray, arities) -> np.ndarray:
    """(sum(arities), m) bool matrix: row soff[v] + s is (D[v] == s)."""
    D = np.asarray(D)
    rows = []
    for v, r in enumerate(np.asarray(arities, dtype=np.int64)):
        for s in range(int(r)):
            rows.append(D[v] == s)
    return np.array(rows, dtype=bool).reshape(len(rows), D.shape[1])


def itemset_support(X: np.ndarray, items) -> int:
    """Transactions holding every item of ``items`` (all m for the empty set)."""
    if len(items) == 0:
        return int(X.shape[1])
    return int(np.logical_and.reduce(X[list(items)], axis=0).sum())


def mine_rules(X: np.ndarray, min_support: float, min_confidence: float, max_size: int,
               all_splits: bool = False, stats: dict | None = None):
    """Frequent itemsets of at most ``max_size`` items and their rules.

    Returns ``(itemsets, supports, rules)``: itemsets as tuples in the order
    described above, their int supports, and rules as (itemset index,
    antecedent mask, confidence in double precision).  When ``stats`` is a
    dict, ``stats["candidates"]`` counts the itemsets of 2 or more items that
    were scanned.
    """
    n_items, m = X.shape
    thr = float(min_support) * float(m)
    freq: dict[tuple, int] = {}
    itemsets: list[tuple] = []
    supports: list[int] = []

    level = []
    if max_size >= 1:
        for i in range(n_items):
            s = itemset_support(X, (i,))
            if float(s) > thr:
                level.append((i,))
                freq[(i,)] = s
    frequent_items = [S[0] for S in level]
    for S in level:
        itemsets.append(S)
        supports.append(freq[S])

    k = 2
    while level and k <= max_size:
        nxt = []
        for S in level:
            for j in frequent_items:
                if j <= S[-1]:
                    continue
                T = S + (j,)
                if not all(T[:t] + T[t + 1:] in freq for t in range(k)):
                    continue
                s = itemset_support(X, T)
                if stats is not None:
                    stats["candidates"] = stats.get("candidates", 0) + 1
                if float(s) > thr:
                    nxt.append(T)
                    freq[T] = s
        for T in nxt:
            itemsets.append(T)
            supports.append(freq[T])
        level = nxt
        k += 1

    rules = []
    for idx, S in enumerate(itemsets):
        k = len(S)
        if k < 2:
            continue
        full = (1 << k) - 1
        for mask in range(1, full):
            if not all_splits and bin(mask).count("1") != k - 1:
                continue
            A = tuple(S[t] for t in range(k) if mask >> t & 1)
            sa = freq[A]
            if float(supports[idx]) > float(min_confidence) * float(sa):
                rules.append((idx, mask, supports[idx] / sa))
    return itemsets, supports, rules
