"""Seeded generators for the synthetic stand-ins of the paper's workloads.

The paper measures on public Bayesian-network benchmark data (Tab. 1) that is
not available here; these generators produce data of the same kind: complete
categorical databases forward-sampled from random DAGs with Dirichlet CPTs,
random query streams drawn without replacement (Sec. 4.1), parent-set score
queries (Sec. 4.2) and binary transactions with skewed item frequencies plus
candidate itemsets (Sec. 4.3).

Conventions shared by every consumer:
  * a database is ``D`` with shape ``(n, m)``, dtype uint8, column ``D[i]`` is
    the paper's ``D_i`` (Sec. 2) and states are stored 0-based (paper: 1..r_i);
  * transaction data is one packed bitmap per item, ``uint64`` words, bit
    ``p % 64`` of word ``p // 64`` set when transaction ``p`` holds the item.

Random numbers come from ``numpy.random.default_rng(seed)`` only.
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np


@dataclasses.dataclass
class Database:
    D: np.ndarray          # (n, m) uint8, column-major: D[i] = states of X_i
    arities: np.ndarray    # (n,) int32
    parents: list          # parents[i] = list of parent variable ids in the DAG
    seed: int

    @property
    def n(self) -> int:
        return int(self.D.shape[0])

    @property
    def m(self) -> int:
        return int(self.D.shape[1])


def random_dag_database(n: int, m: int, arity_lo: int, arity_hi: int,
                        max_indeg: int, alpha: float, seed: int,
                        chunk: int = 1 << 20) -> Database:
    """Forward-sample ``m`` instances from a random DAG over ``n`` variables.

    Recipe: a random topological order; the node at position t draws its
    in-degree uniformly from {0..min(max_indeg, t)} and its parents uniformly
    among earlier nodes; arities are uniform in {arity_lo..arity_hi}; each
    parent configuration gets one CPT row drawn from Dirichlet(alpha * 1_r);
    instances are sampled node by node in topological order.
    """
    rng = np.random.default_rng(seed)
    arities = rng.integers(arity_lo, arity_hi + 1, size=n).astype(np.int32)
    order = rng.permutation(n)
    parents = [[] for _ in range(n)]
    cpts = [None] * n
    for t, v in enumerate(order):
        d = int(rng.integers(0, min(max_indeg, t) + 1))
        pa = sorted(int(x) for x in rng.choice(order[:t], size=d, replace=False)) if d else []
        parents[v] = pa
        q = int(np.prod([arities[p] for p in pa])) if pa else 1
        cpts[v] = rng.dirichlet(np.full(int(arities[v]), alpha), size=q)
    D = np.empty((n, m), dtype=np.uint8)
    for lo in range(0, m, chunk):
        hi = min(m, lo + chunk)
        for v in order:
            pa = parents[v]
            cum = np.cumsum(cpts[v], axis=1)
            u = rng.random(hi - lo)
            s = np.zeros(hi - lo, dtype=np.uint8)
            if pa:
                row = np.zeros(hi - lo, dtype=np.int32)
                for p in pa:  # index of the CPT row used by each instance
                    row = row * int(arities[p]) + D[p, lo:hi]
                for j in range(int(arities[v]) - 1):  # inverse-CDF draw
                    s += u >= cum[:, j][row]
            else:
                for j in range(int(arities[v]) - 1):
                    s += u >= cum[0, j]
            D[v, lo:hi] = s
    return Database(D=D, arities=arities, parents=parents, seed=seed)


def subset_queries(n: int, sizes) -> list:
    """Every variable subset of the given sizes, ascending ids (config: tiny)."""
    out = []
    for k in sizes:
        out.extend(list(c) for c in itertools.combinations(range(n), k))
    return out


def random_queries(n: int, nq: int, k_lo: int, k_hi: int, seed: int) -> list:
    """``nq`` queries, size uniform in {k_lo..k_hi}, variables drawn uniformly
    without replacement (the random-query protocol of Sec. 4.1)."""
    rng = np.random.default_rng(seed)
    ks = rng.integers(k_lo, k_hi + 1, size=nq)
    return [[int(x) for x in rng.choice(n, size=int(k), replace=False)] for k in ks]


def score_queries(n: int, nq: int, pa_lo: int, pa_hi: int, seed: int):
    """``nq`` (child, parents) pairs, |parents| uniform in {pa_lo..pa_hi},
    parents distinct and different from the child (Sec. 4.2 query form)."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(pa_lo, pa_hi + 1, size=nq)
    child, parents = [], []
    for s in sizes:
        pick = rng.choice(n, size=int(s) + 1, replace=False)
        child.append(int(pick[0]))
        parents.append([int(x) for x in pick[1:]])
    return child, parents


def zipf_item_probs(n_items: int, s: float, mean_len: float) -> np.ndarray:
    """Item inclusion probabilities p_i = min(1, c * i^-s), i = 1..n_items, with
    c chosen by bisection so that sum(p_i) = mean_len."""
    i = np.arange(1, n_items + 1, dtype=np.float64)
    w = i ** (-s)
    lo, hi = 0.0, float(mean_len) / float(w.min())
    for _ in range(200):
        c = 0.5 * (lo + hi)
        if np.minimum(1.0, c * w).sum() < mean_len:
            lo = c
        else:
            hi = c
    return np.minimum(1.0, 0.5 * (lo + hi) * w)


def zipf_transaction_bitmaps(n_items: int, m: int, s: float, mean_len: float,
                             seed: int) -> np.ndarray:
    """Independent Bernoulli(p_i) inclusion of item i in each of ``m``
    transactions, returned as packed bitmaps of shape (n_items, ceil(m/64)),
    uint64.  Set positions are drawn as a Bernoulli process by geometric gaps."""
    rng = np.random.default_rng(seed)
    p = zipf_item_probs(n_items, s, mean_len)
    words = (m + 63) // 64
    out = np.zeros((n_items, words), dtype=np.uint64)
    mask = np.zeros(words * 64, dtype=bool)
    for it in range(n_items):
        mask[:] = False
        pi = float(p[it])
        if pi >= 1.0:
            mask[:m] = True
        elif pi > 0.0:
            pos = np.empty(0, dtype=np.int64)
            last = -1
            while True:
                need = max(16, int((m - last) * pi * 1.05 + 6 * np.sqrt(m * pi) + 16))
                gaps = rng.geometric(pi, size=need)
                cand = last + np.cumsum(gaps)
                pos = np.concatenate([pos, cand[cand < m]])
                if cand[-1] >= m:
                    break
                last = int(cand[-1])
            mask[pos] = True
        out[it] = np.packbits(mask, bitorder="little").view(np.uint64)
    return out


def basket_transaction_bitmaps(n_items: int, m: int, n_groups: int, seed: int) -> np.ndarray:
    """Correlated transactions: item i belongs to group i % n_groups; each
    transaction switches group g on with probability a_g ~ U(0.3, 0.8); an
    item is present with probability p_i ~ U(0.6, 0.95) when its group is on
    and e_i ~ U(0, 0.15) otherwise.  Items of one group therefore co-occur and
    form frequent itemsets of several items.  Packed like
    zipf_transaction_bitmaps: shape (n_items, ceil(m/64)), uint64, bit p of
    word w is transaction 64 w + p."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.3, 0.8, size=n_groups)
    p_on = rng.uniform(0.6, 0.95, size=n_items)
    p_off = rng.uniform(0.0, 0.15, size=n_items)
    words = (m + 63) // 64
    out = np.zeros((n_items, words), dtype=np.uint64)
    on = rng.random((n_groups, m)) < a[:, None]
    row = np.zeros(words * 64, dtype=bool)
    for it in range(n_items):
        g = it % n_groups
        u = rng.random(m)
        row[:m] = np.where(on[g], u < p_on[it], u < p_off[it])
        out[it] = np.packbits(row, bitorder="little").view(np.uint64)
    return out


def weighted_itemsets(n_items: int, nq: int, k_lo: int, k_hi: int,
                      probs: np.ndarray, seed: int) -> list:
    """``nq`` distinct itemsets, size uniform in {k_lo..k_hi}; items within a
    set are drawn by successive sampling without replacement with probability
    proportional to ``probs`` (a redraw on collision is exactly a draw from the
    weights restricted to the items not yet chosen).  Items are returned sorted."""
    rng = np.random.default_rng(seed)
    cdf = np.cumsum(probs / probs.sum())
    cdf[-1] = 1.0
    sizes = rng.integers(k_lo, k_hi + 1, size=nq)
    seen = set()
    out = [None] * nq
    for k in range(k_lo, k_hi + 1):
        slots = np.nonzero(sizes == k)[0]
        fill = 0
        stalled = 0
        while fill < len(slots):
            before = fill
            want = len(slots) - fill
            batch = max(64, int(want * 1.2))
            draws = np.empty((batch, k), dtype=np.int64)
            for t in range(k):
                col = np.searchsorted(cdf, rng.random(batch), side="right")
                while True:
                    clash = np.zeros(batch, dtype=bool)
                    for u in range(t):
                        clash |= draws[:, u] == col
                    if not clash.any():
                        break
                    col[clash] = np.searchsorted(cdf, rng.random(int(clash.sum())), side="right")
                draws[:, t] = col
            draws.sort(axis=1)
            for row in draws:
                key = tuple(int(x) for x in row)
                if key in seen:
                    continue
                seen.add(key)
                out[slots[fill]] = list(key)
                fill += 1
                if fill == len(slots):
                    break
            stalled = stalled + 1 if fill == before else 0
            if stalled > 50:
                raise ValueError(f"cannot draw {len(slots)} distinct itemsets of size {k} "
                                 f"from {n_items} items")
    return out


# The five workload shapes.  ``data`` gives the database recipe, ``queries``
# the query stream; sizes are those of the benchmark configurations.
CONFIGS = {
    "tiny": dict(n=8, m=1000, arity=(2, 4), max_indeg=2, alpha=1.0, seed=1),
    "random": dict(n=40, m=100_000, arity=(2, 5), max_indeg=3, alpha=0.5, seed=2,
                   nq=10_000, k=(2, 6)),
    "pairs": dict(n=256, m=1_000_000, arity=(2, 3), max_indeg=2, alpha=0.5, seed=3),
    "scores": dict(n=64, m=1_000_000, arity=(2, 4), max_indeg=4, alpha=1.0, seed=4,
                   nq=50_000, pa=(0, 4), ess=1.0),
    "support": dict(n_items=1000, m=10_000_000, zipf_s=1.1, mean_len=10.0, seed=5,
                    nq=1_000_000, k=(2, 5)),
    # the same itemsets with every antecedent split (2^k - 2 rules each)
    "splits": dict(n_items=1000, m=10_000_000, zipf_s=1.1, mean_len=10.0, seed=5,
                   nq=1_000_000, k=(2, 5)),
    # the parent-set lattice over the first 20 variables of the BN-score
    # database, parent sets of at most 4 (Sec. 4.2 query stream)
    "families": dict(m=1_000_000, nv=20, max_parents=4, seed=4),
    # streaming appends: the BN-score database loaded with 1e6 instances, then
    # grown by blocks of 1e6 instances (Sec. 6)
    "append": dict(m=1_000_000, block=1_000_000),
    # bottom-up rule mining over the (variable, state) items of the BN-score
    # database: support > 0.2, confidence > 0.3, itemsets of at most 6 items
    # (Sec. 4.3 thresholds), single-item consequents
    "rules": dict(m=1_000_000, min_support=0.2, min_confidence=0.3, max_size=6),
    # specific assignments over the batched-random database (end of Sec. 3.3)
    "assign": dict(m=100_000, seed=7, nq=100_000, k=(1, 6)),
    # tables beyond shared memory (up to 16^5 cells): the global-atomic and
    # sort + run-length paths
    "large": dict(n=8, m=1_000_000, arity=(12, 16), max_indeg=2, alpha=0.3, seed=6,
                  nq=64, k=(4, 5)),
}


def config_database(name: str, m: int | None = None) -> Database:
    """Database of one of the categorical workloads, optionally with fewer rows."""
    c = CONFIGS[name]
    return random_dag_database(c["n"], c["m"] if m is None else m, c["arity"][0],
                               c["arity"][1], c["max_indeg"], c["alpha"], c["seed"])
