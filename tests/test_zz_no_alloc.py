"""The allocation-free entry point fc_count_sorted_noalloc against fc_count.

Some callers cannot let a library allocate device memory: a global-mode
stream capture refuses cudaMalloc, some programs own all device memory through
their own pool allocator, and latency-critical paths avoid the device
synchronisation that cudaMalloc and cudaFree may cause.  For them the library
offers one sort + run-length count whose scratch is a fixed array compiled
into the library.  These tests compare its tables with the regular fc_count
on the same data, on calls made one after the other (they share that scratch,
which keeps the previous call's contents).  Counts must agree exactly.
"""
import numpy as np
import pytest

import paper_1804_04640_gb300 as fc
from workloads import random_dag_database

pytestmark = pytest.mark.gpu


def _cells(arities, q):
    out = 1
    for v in q:
        out *= int(arities[v])
    return out


def test_noalloc_matches_fc_count_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    fc.load_library(build_if_missing=True)
    db = random_dag_database(12, 300_007, 2, 6, 3, 0.5, seed=91)
    ctx = fc.fc_load(db.D, db.arities)
    # column-major rows with a leading dimension larger than m
    wide = torch.zeros((db.n, db.m + 100), dtype=torch.uint8, device="cuda")
    wide[:, : db.m] = torch.from_numpy(db.D).cuda()
    D = wide[:, : db.m]
    stream = torch.cuda.current_stream()
    for q in ([0, 3, 5], [7, 1, 2, 9, 11], [0, 3, 5], [4]):
        out = torch.full((_cells(db.arities, q),), -1, dtype=torch.int32, device="cuda")
        fc.fc_count_sorted_noalloc(D, db.arities, q, out, stream)
        torch.cuda.synchronize()
        want = fc.fc_count(ctx, q)
        assert np.array_equal(out.cpu().numpy(), want), q


def test_noalloc_rejects_too_many_instances():
    torch = pytest.importorskip("torch")
    fc.load_library(build_if_missing=True)
    big = torch.zeros((2, (1 << 20) + 1), dtype=torch.uint8, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(fc.FcError) as e:
        fc.fc_count_sorted_noalloc(big, [2, 2], [0, 1], out)
    assert e.value.code == fc.FC_ERR_SIZE
    assert "at most" in fc.fc_last_error()
