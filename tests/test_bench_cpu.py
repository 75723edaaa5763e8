"""The benchmark's JSON contract on the CPU: the roofline object of every
workload, the workload description both arms print, and the batch split
across ranks (no GPU needed: these are the bench's own host functions)."""
import math

import pytest

import bench

PK = {"hbm_gbs": 6789.6, "bf16_tflops": 1887.8, "src": "measured", "l2_read_gbs_4mib": 21500.0,
      "l2_read_gbs_64mib": 19400.0, "smem_atomics_g_per_s": 9850.0, "and_popc_g_words_per_s": 2490.0}

WORK = {"atomics": 10 ** 9, "col_bytes": 4 * 10 ** 9, "alg_bytes": 4 * 10 ** 9, "keyed_queries": 10_000,
        "queries": 10_000, "flops": 4.15e11, "popc_words": 2 * 10 ** 12}

BOUNDS = {"tiny": "smem_atomic", "random": "smem_atomic", "large": "smem_atomic", "scores": "smem_atomic",
          "pairs": "tensor", "support": "alu", "splits": "alu", "assign": "alu", "families": "l2",
          "rules": "l2", "append": "hbm"}


@pytest.mark.parametrize("name", sorted(BOUNDS))
def test_roofline_object_of_every_workload(name):
    resident = 2 * bench.L2_BYTES if name in ("support", "splits", "append") else 4 << 20
    r = bench.roofline(name, 0.5, WORK, PK, resident, "-")
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in r, key
    assert r["bound"] == BOUNDS[name]
    assert math.isclose(r["frac"], r["achieved"] / r["peak"])
    # achieved = the step's work over its time, in the unit's scale
    if name == "pairs":
        assert math.isclose(r["achieved"], WORK["flops"] / 0.5e-3 / 1e12)
        assert math.isclose(r["peak"], 2 * PK["bf16_tflops"])
    elif r["bound"] == "smem_atomic":
        assert math.isclose(r["achieved"], WORK["atomics"] / 0.5e-3 / 1e9)
        assert math.isclose(r["l2"]["frac"], WORK["col_bytes"] / 0.5e-3 / 1e9 / PK["l2_read_gbs_4mib"])
    elif r["bound"] == "alu":
        assert math.isclose(r["achieved"], WORK["popc_words"] / 0.5e-3 / 1e9)


def test_traffic_is_keyed_to_the_plan():
    # a plan signature that no capture recorded reports no traffic
    assert bench.measured_traffic("random", "hist=1") is None
    assert bench.measured_traffic("no-such-workload", "-") is None


def test_both_arms_describe_the_same_workload():
    """The GPU arm and the reference arm build the workload the same way and
    print the same config dict (tiny: the default run's first nested config)."""
    w1 = bench.make_workload("tiny")
    w2 = bench.make_workload("tiny")
    assert bench.describe("tiny", w1) == bench.describe("tiny", w2)
    c = bench.describe("tiny", w1)
    assert set(c) == {"workload", "n", "m", "queries"}
    assert c["queries"] == 92 and c["m"] == 1000


@pytest.mark.parametrize("world", [1, 2, 3])
def test_rank_slices_tile_the_job_batch(world):
    """A query workload at `world` ranks draws world x nq queries and every
    rank takes a contiguous slice; the slices are the whole batch, once."""
    parts = [bench.make_workload("random", m=4096, nq=30, rank=r, world=world)["queries"] for r in range(world)]
    whole = bench.make_workload("random", m=4096, nq=30 * world)["queries"]
    assert sum(parts, []) == whole
    assert all(len(p) == 30 for p in parts)


def test_oracle_family_enumeration():
    fams = bench.oracle_families([0, 1, 2, 3], 2)
    # each child with every parent set of <= 2 of the other three: 1 + 3 + 3
    assert len(fams) == 4 * 7
    assert (0, []) in fams and (3, [0, 1]) in fams and (1, [0, 2]) in fams
    assert all(c not in pa for c, pa in fams)


def test_options_are_echoed_only_when_given():
    """--option settings appear under config.options; without them the GPU
    arm's config is the reference arm's (describe) unchanged."""
    import argparse
    w = bench.make_workload("tiny")
    base = bench.describe("tiny", w)
    assert bench.with_options(base, argparse.Namespace(option=[])) == base
    got = bench.with_options(base, argparse.Namespace(option=["codes4=0", "device_plan=1"]))
    assert got["options"] == ["codes4=0", "device_plan=1"]
    assert {k: v for k, v in got.items() if k != "options"} == base
