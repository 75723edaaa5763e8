"""The allocation-free entry point fc_count_sorted_noalloc.

Some callers cannot let a library allocate device memory: a global-mode
stream capture refuses cudaMalloc, some programs own all device memory through
their own pool allocator, and latency-critical paths avoid the device
synchronisation that cudaMalloc and cudaFree may cause.  For them the library
offers one sort + run-length count whose scratch is a fixed array compiled
into the library.  These tests compare its tables with the regular fc_count
and with the CPU oracle on the same data, on calls made one after the other
(they share that scratch, which keeps the previous call's contents).  Counts
must agree exactly.  The file is collected last so that a run that stops at
its first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
import paper_1804_04640_gb300 as fc
from workloads import random_dag_database

pytestmark = pytest.mark.gpu


def _cells(arities, q):
    out = 1
    for v in q:
        out *= int(arities[v])
    return out


def test_noalloc_matches_fc_count_and_oracle_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    fc.load_library(build_if_missing=True)
    db = random_dag_database(12, 300_007, 2, 6, 3, 0.5, seed=91)
    ctx = fc.fc_load(db.D, db.arities)
    orc = oracle.DB(db.D, db.arities)
    # column-major rows with a leading dimension larger than m
    wide = torch.zeros((db.n, db.m + 100), dtype=torch.uint8, device="cuda")
    wide[:, : db.m] = torch.from_numpy(db.D).cuda()
    D = wide[:, : db.m]
    stream = torch.cuda.current_stream()
    for q in ([0, 3, 5], [7, 1, 2, 9, 11], [0, 3, 5], [4], [], [10, 8, 6, 4, 2, 0]):
        out = torch.full((_cells(db.arities, q),), -1, dtype=torch.int32, device="cuda")
        fc.fc_count_sorted_noalloc(D, db.arities, q, out, stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, fc.fc_count(ctx, q)), q
        assert np.array_equal(got.astype(np.int64), orc.table(q)), q


@pytest.mark.parametrize("arity,k", [(16, 2), (16, 3), (2, 8)])
def test_noalloc_drops_instances_with_states_outside_the_arity(arity, k):
    """An instance whose state of a queried variable is >= its arity gets a
    key with every bit set and is not counted.  With 256 cells (16 x 16 and
    2^8) the single 8-bit sort pass leaves those keys in the same bucket as
    cell 255, interleaved with its instances; 4096 cells take two passes."""
    torch = pytest.importorskip("torch")
    fc.load_library(build_if_missing=True)
    rng = np.random.default_rng(1000 + arity * 10 + k)
    n, m = k + 1, 200_003
    arities = np.full(n, arity, dtype=np.int32)
    D = rng.integers(0, arity, size=(n, m)).astype(np.uint8)
    # a third of the instances sit in the last cell, so its runs are long
    last = rng.random(m) < 0.33
    D[:k, last] = arity - 1
    # 5% of the instances get a state past the arity in one queried variable
    bad = rng.random(m) < 0.05
    which = rng.integers(0, k, size=m)
    D[which[bad], np.nonzero(bad)[0]] = rng.integers(arity, 256, size=int(bad.sum())).astype(np.uint8)
    q = list(range(k))
    good = np.all(D[:k] < arity, axis=0)
    want = oracle.DB(np.ascontiguousarray(D[:, good]), arities).table(q)
    Dd = torch.from_numpy(D).cuda()
    for _ in range(2):  # two calls in a row share the scratch
        out = torch.full((_cells(arities, q),), -7, dtype=torch.int32, device="cuda")
        fc.fc_count_sorted_noalloc(Dd, arities, q, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().astype(np.int64), want)


def test_noalloc_with_no_instances_gives_zeros():
    torch = pytest.importorskip("torch")
    fc.load_library(build_if_missing=True)
    D = torch.zeros((3, 0), dtype=torch.uint8, device="cuda")
    out = torch.full((2 * 3 * 4,), 5, dtype=torch.int32, device="cuda")
    fc.fc_count_sorted_noalloc(D, [2, 3, 4], [0, 1, 2], out)
    torch.cuda.synchronize()
    assert not out.cpu().numpy().any()


def test_noalloc_rejects_too_many_instances():
    torch = pytest.importorskip("torch")
    fc.load_library(build_if_missing=True)
    big = torch.zeros((2, (1 << 20) + 1), dtype=torch.uint8, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(fc.FcError) as e:
        fc.fc_count_sorted_noalloc(big, [2, 2], [0, 1], out)
    assert e.value.code == fc.FC_ERR_SIZE
    assert "at most" in fc.fc_last_error()


def test_noalloc_refuses_bad_buffers_before_any_launch():
    """Buffers the C call cannot check are refused by the binding."""
    torch = pytest.importorskip("torch")
    fc.load_library(build_if_missing=True)
    D = torch.zeros((3, 1000), dtype=torch.uint8, device="cuda")
    ok = torch.zeros(24, dtype=torch.int32, device="cuda")
    cases = [
        (D, [2, 3, 4], [0, 1, 2], torch.zeros(23, dtype=torch.int32, device="cuda"), fc.FC_ERR_SIZE),
        (D, [2, 3, 4], [0, 1, 2], torch.zeros(24, dtype=torch.int64, device="cuda"), fc.FC_ERR_ARG),
        (D, [2, 3, 4], [0, 1, 2], torch.zeros(48, dtype=torch.int32, device="cuda")[::2], fc.FC_ERR_ARG),
        (D.to(torch.int32), [2, 3, 4], [0, 1, 2], ok, fc.FC_ERR_ARG),
        (D.t().contiguous().t(), [2, 3, 4], [0, 1, 2], ok, fc.FC_ERR_ARG),
        (D, [2, 3], [0, 1], ok, fc.FC_ERR_ARG),
        (D, [2, 3, 4], [0, 3], ok, fc.FC_ERR_ARG),
    ]
    for Dx, ar, q, out, code in cases:
        with pytest.raises(fc.FcError) as e:
            fc.fc_count_sorted_noalloc(Dx, ar, q, out)
        assert e.value.code == code
