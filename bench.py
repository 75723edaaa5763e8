#!/usr/bin/env python3
"""Benchmark of the counting-query hot path on GB300.

Default workload ("random"): n = 40 categorical variables (arity 2-5),
m = 100,000 instances sampled from a random DAG, and a batch of 10,000 queries
of 2-6 variables drawn without replacement.  One step answers the whole batch
(every full contingency table) with one graph launch of the persistent count
kernel.  Printed as one JSON line:

  value         queries/s, device-resident inputs and outputs (max over ranks);
  e2e           the same through fc_count_batch with pinned host buffers
                (planning, host-to-device descriptors, kernel, device-to-host tables);
  per_query     the same queries issued as one launch each;
  roofline      the step's work over its time against the measured rate of the
                unit that bounds the dominant kernel (probe rates measured at
                start-up by fc_probe_rate, listed under probe_peaks);
  cpu_baseline  the CPU oracle on a bounded sample, on this host's cores;
  clocks        SM clock and throttle reasons sampled while the GPU works;
  configs       (one GPU, default run) the other benchmark configurations --
                tiny, pairs, scores, support -- each with its own value,
                roofline, e2e, cpu_baseline and clocks.

Other workloads (--workload ...) print their own line.  `--impl reference`
times the CPU oracle on the same workload.  With --gpus N > 1 (one rank per
GPU; a bare `bench.py --gpus N` relaunches itself under torchrun) every rank
answers its own slice of a batch of N x the workload's queries.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import (CONFIGS, config_database, random_dag_database, random_queries,  # noqa: E402
                       score_queries, subset_queries, weighted_itemsets, zipf_item_probs,
                       zipf_transaction_bitmaps)

L2_BYTES = 129 * 2**20


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", 0)), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


def measured_traffic(workload: str, plan_sig: str):
    """DRAM bytes per launch of the workload's dominant kernel from the committed
    ncu summary, or None when the kernel source or the plan (the strategy mix
    of a count workload) changed since the capture."""
    import hashlib
    try:
        lines = open(os.path.join(ROOT, "profiles", "traffic.txt")).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        parts = ln.split()
        if len(parts) != 6 or ln.startswith("#") or parts[0] != workload or parts[4] != plan_sig:
            continue
        src = os.path.join(ROOT, "paper_1804_04640_gb300", "csrc", parts[2])
        try:
            sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        except OSError:
            return None
        return int(parts[5]) if sha == parts[3] else None
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock, utilisation and throttle reasons while
    the GPU works (started before the warm-up, stopped before the CPU legs)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.proc = None

    def __exit__(self, *a):
        self.stop()

    def summary(self):
        sm, mx, busy, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            try:
                if float(parts[3]) >= 50:
                    busy.append(sm[-1])
            except ValueError:
                pass
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "samples_busy": len(busy),
                "window": "warm-up, timed steps, per-query and end-to-end legs (50 ms period)"}


# ------------------------------------------------------------------ workloads

def _database(name: str, m: int | None, rank: int):
    """The workload's database; rank r > 0 of a multi-rank job draws its own
    (seed + 1000 r) where ranks solve independent problems."""
    if rank == 0:
        return config_database(name, m)
    c = CONFIGS[name]
    return random_dag_database(c["n"], c["m"] if m is None else m, c["arity"][0], c["arity"][1],
                               c["max_indeg"], c["alpha"], c["seed"] + 1000 * rank)


def make_workload(name: str, m: int | None = None, nq: int | None = None, rank: int = 0, world: int = 1):
    """Seeded inputs of one workload (host arrays); m / nq shrink it (profiling).

    With world > 1 ranks, a query workload draws one batch of world x nq
    queries (the database is replicated) and each rank takes its own slice
    (shard.split_batch), so every query is answered once; the workloads
    without a query batch give every rank its own database instead."""
    from paper_1804_04640_gb300 import shard

    c = dict(CONFIGS[name])
    if m:
        c["m"] = m
    if nq:
        c["nq"] = nq
    gq = c.get("nq", 0) * world  # queries of the whole job

    def part(batch):
        return shard.split_batch(batch, rank, world)

    if name in ("tiny", "random", "large"):
        if name == "tiny":
            db = _database(name, c["m"], rank)
            queries = subset_queries(db.n, (1, 2, 3))
        else:
            db = config_database(name, c["m"])
            queries = part(random_queries(db.n, gq, c["k"][0], c["k"][1], c["seed"]))
        return {"db": db, "queries": queries}
    if name == "families":
        db = _database("scores", c["m"], rank)
        return {"db": db, "vars": list(range(c["nv"])), "max_parents": c["max_parents"]}
    if name == "rules":
        return {"db": _database("scores", c["m"], rank), "args": (c["min_support"], c["min_confidence"],
                                                                  c["max_size"], False)}
    if name == "append":
        return {"db": _database("scores", c["m"] + c["block"], rank), "m0": c["m"], "block": c["block"]}
    if name == "assign":
        db = config_database("random", c["m"])
        rng = np.random.default_rng(c["seed"])
        qs = []
        for _ in range(gq):
            k = int(rng.integers(c["k"][0], c["k"][1] + 1))
            vs = [int(x) for x in rng.choice(db.n, size=k, replace=False)]
            qs.append((vs, [int(rng.integers(0, db.arities[v])) for v in vs]))
        return {"db": db, "assign": part(qs)}
    if name == "scores":
        db = config_database(name, c["m"])
        child, parents = score_queries(db.n, gq, c["pa"][0], c["pa"][1], c["seed"])
        return {"db": db, "child": part(child), "parents": part(parents)}
    if name == "pairs":
        return {"db": _database(name, c["m"], rank)}
    if name in ("support", "splits"):
        bits = zipf_transaction_bitmaps(c["n_items"], c["m"], c["zipf_s"], c["mean_len"], c["seed"])
        probs = zipf_item_probs(c["n_items"], c["zipf_s"], c["mean_len"])
        sets = weighted_itemsets(c["n_items"], gq, c["k"][0], c["k"][1], probs, c["seed"])
        return {"bits": bits, "m": c["m"], "sets": part(sets)}
    raise ValueError(name)


def with_options(config: dict, args) -> dict:
    """The workload description plus any --option settings the run used."""
    if getattr(args, "option", None):
        config = dict(config, options=list(args.option))
    return config


def describe(name: str, w) -> dict:
    c = CONFIGS[name]
    if name in ("tiny", "random", "large"):
        ks = [len(q) for q in w["queries"]]
        return {"workload": f"{name}: n={w['db'].n} arity {c['arity'][0]}-{c['arity'][1]}, m={w['db'].m}, "
                            f"{len(ks)} count queries of {min(ks)}-{max(ks)} variables",
                "n": w["db"].n, "m": w["db"].m, "queries": len(ks)}
    if name == "families":
        nf = len(w["vars"])
        return {"workload": f"families: BN-score database (n={w['db'].n}, m={w['db'].m}), every child of the "
                            f"first {nf} variables with every parent set of <= {w['max_parents']} of the others, BDeu",
                "n": w["db"].n, "m": w["db"].m, "variables": nf, "max_parents": w["max_parents"]}
    if name == "append":
        return {"workload": f"append: BN-score database (n={w['db'].n}) loaded with {w['m0']} instances, "
                            f"each step appends a block of {w['block']} instances from device memory",
                "n": w["db"].n, "m0": w["m0"], "block": w["block"]}
    if name == "rules":
        a = w["args"]
        return {"workload": f"rules: bottom-up mining over the {int(w['db'].arities.sum())} (variable, state) items "
                            f"of the BN-score database (n={w['db'].n}, m={w['db'].m}), support > {a[0]}, "
                            f"confidence > {a[1]}, itemsets of <= {a[2]} items, single-item consequents",
                "n": w["db"].n, "m": w["db"].m, "min_support": a[0], "min_confidence": a[1], "max_size": a[2]}
    if name == "assign":
        return {"workload": f"assign: n={w['db'].n}, m={w['db'].m}, {len(w['assign'])} specific assignments of "
                            f"{c['k'][0]}-{c['k'][1]} conditions", "n": w["db"].n, "m": w["db"].m,
                "queries": len(w["assign"])}
    if name == "scores":
        return {"workload": f"scores: n={w['db'].n}, m={w['db'].m}, {len(w['child'])} (child, parents) "
                            f"queries, |parents| {c['pa'][0]}-{c['pa'][1]}, MDL and BDeu(ess=1)",
                "n": w["db"].n, "m": w["db"].m, "queries": len(w["child"])}
    if name == "pairs":
        n = w["db"].n
        return {"workload": f"pairs: n={n}, m={w['db'].m}, all {n * (n - 1) // 2} pairwise tables + MI",
                "n": n, "m": w["db"].m, "sum_arity": int(w["db"].arities.sum())}
    what = ("supports + supports and confidences of every antecedent split (2^k - 2 rules each)"
            if name == "splits" else "supports + single-consequent rule confidences")
    return {"workload": f"{name}: {len(w['bits'])} items, m={w['m']}, {len(w['sets'])} itemsets of "
                        f"{c['k'][0]}-{c['k'][1]} items, {what}",
            "n_items": len(w["bits"]), "m": w["m"], "queries": len(w["sets"])}


# ------------------------------------------------------------ CPU oracle arm

def oracle_families(vars_, max_parents: int):
    """(child, parents) of every family over `vars_` with at most `max_parents`
    parents drawn from the other variables (the oracle leg's own enumeration)."""
    import itertools
    vs = [int(x) for x in vars_]
    out = []
    for c in vs:
        rest = [v for v in vs if v != c]
        for d in range(min(max_parents, len(rest)) + 1):
            out.extend((c, list(pa)) for pa in itertools.combinations(rest, d))
    return out


def oracle_rate(name: str, w, seconds: float, cores: int):
    """Units/s of the CPU oracle (as it stands) on a bounded sample."""
    import oracle

    units = 0
    sample = ""
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        if name in ("tiny", "random", "large", "scores"):
            orc = oracle.DB(w["db"].D, w["db"].arities)
            if name == "scores":
                jobs = [(w["child"][q], w["parents"][q]) for q in range(len(w["child"]))]
                def fn(j):
                    orc.score(j[0], j[1], "mdl")
                    return orc.score(j[0], j[1], "bdeu")
            else:
                jobs = w["queries"]
                fn = orc.table
            t0 = time.perf_counter()
            i = 0
            while time.perf_counter() - t0 < seconds:
                chunk = jobs[i % len(jobs): i % len(jobs) + 4 * cores] or jobs[: 4 * cores]
                list(ex.map(fn, chunk))
                units += len(chunk)
                i += len(chunk)
            sample = f"{units} queries of the workload (in order, wrapping), {cores} threads"
        elif name == "families":
            orc = oracle.DB(w["db"].D, w["db"].arities)
            jobs = oracle_families(w["vars"], w["max_parents"])
            t0 = time.perf_counter()
            i = 0
            while time.perf_counter() - t0 < seconds:
                chunk = jobs[i % len(jobs): i % len(jobs) + 4 * cores] or jobs[: 4 * cores]
                list(ex.map(lambda f: orc.score(f[0], f[1], "bdeu"), chunk))
                units += len(chunk)
                i += len(chunk)
            sample = f"{units} families scored one by one from row scans, {cores} threads"
        elif name == "append":
            # the oracle has no incremental state: a grown database is scanned
            # again, so its append rate is the rate of re-deriving the
            # marginals (one pass over every instance) per appended block
            db = w["db"]
            orc = oracle.DB(db.D[:, : w["m0"] + w["block"]], db.arities)
            t0 = time.perf_counter()
            rows = 0
            while rows == 0 or time.perf_counter() - t0 < seconds:
                for v in range(db.n):
                    orc.table([v])
                rows += w["block"]
            dt_s = time.perf_counter() - t0
            return rows / dt_s, (f"one-variable tables of all {db.n} variables over the "
                                 f"{w['m0'] + w['block']} instances after an append, repeated, 1 thread")
        elif name == "rules":
            from oracle import miner
            db = w["db"]
            ms = max(1000, min(db.m, 20_000))
            X = miner.item_matrix_from_db(db.D[:, :ms], db.arities)
            st = {}
            t0 = time.perf_counter()
            miner.mine_rules(X, *w["args"], stats=st)
            dt_s = time.perf_counter() - t0
            # the row scans dominate and grow linearly in m: scale to the full rows
            units = st.get("candidates", 0) * ms / db.m
            sample = (f"the whole mining run on the first {ms} of {db.m} rows ({st.get('candidates', 0)} candidates "
                      f"scanned in {dt_s:.1f} s, 1 thread), rate scaled by {ms}/{db.m}")
            return units / dt_s, sample
        elif name == "assign":
            orc = oracle.DB(w["db"].D, w["db"].arities)
            jobs = w["assign"]
            t0 = time.perf_counter()
            i = 0
            while time.perf_counter() - t0 < seconds:
                chunk = jobs[i % len(jobs): i % len(jobs) + 4 * cores] or jobs[: 4 * cores]
                list(ex.map(lambda q: orc.count_assignment(*q), chunk))
                units += len(chunk)
                i += len(chunk)
            sample = f"{units} assignments of the workload by row scan, {cores} threads"
        elif name == "pairs":
            orc = oracle.DB(w["db"].D, w["db"].arities)
            n = w["db"].n
            pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
            ar = w["db"].arities
            def fn(p):
                t = orc.table(list(p))
                return oracle.score_table(t, int(ar[p[0]]), int(ar[p[1]]), "mi")
            t0 = time.perf_counter()
            i = 0
            while time.perf_counter() - t0 < seconds:
                chunk = pairs[i: i + 4 * cores] or pairs[: 4 * cores]
                list(ex.map(fn, chunk))
                units += len(chunk)
                i += len(chunk)
            sample = f"{units} pair tables + MI by row scan, {cores} threads"
        else:
            bits, m, sets = w["bits"], w["m"], w["sets"]
            ofn = oracle.support_splits if name == "splits" else oracle.support_rules
            def fn(s):
                return ofn(bits, m, s)
            t0 = time.perf_counter()
            i = 0
            while time.perf_counter() - t0 < seconds:
                chunk = sets[i: i + cores] or sets[:cores]
                list(ex.map(fn, chunk))
                units += len(chunk)
                i += len(chunk)
            what = "every antecedent split" if name == "splits" else "support + k leave-one-out supports"
            sample = f"{units} itemsets ({what}) by transaction scan, {cores} threads"
    dt = time.perf_counter() - t0
    return units / dt, sample


METRIC = "count queries/s (exact full contingency tables, batched persistent launch)"
UNITS = {"tiny": "queries/s", "random": "queries/s", "large": "queries/s", "scores": "queries/s",
         "pairs": "pairs/s", "support": "itemsets/s", "assign": "assignments/s", "families": "families/s",
         "rules": "candidate itemsets/s", "append": "instances/s", "splits": "itemsets/s"}
# the benchmark configurations measured beside the headline by a default run
NESTED = ("tiny", "pairs", "scores", "support")
STRATEGY_NAMES = ["bitmap", "hist", "gatomic", "sort", "marginal", "window"]


def metric_of(name: str) -> str:
    return METRIC if name == "random" else f"{name}: {UNITS[name]}"


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    w = make_workload(args.workload, args.m, args.nq)
    cores = os.cpu_count() or 1
    rate, sample = oracle_rate(args.workload, w, args.ref_seconds, cores)
    if args.workload in ("rules", "append"):
        cores = 1  # these oracle legs run on one thread
    k = args.steps if args.steps is not None else 20
    # each step a bounded sample, the whole run about a minute at most
    per_step = max(0.05, min(args.ref_seconds / 4, 60.0 / max(1, args.warmup + k)))
    steps = []
    for _ in range(args.warmup + k):
        steps.append(oracle_rate(args.workload, w, per_step, cores)[0])
    value = statistics.median(steps[args.warmup:]) if k else rate
    unit = UNITS[args.workload]
    line = {"impl": "reference", "metric": metric_of(args.workload),
            "value": value, "unit": unit, "n_gpus": world, "steps": k, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64/f64",
            "data": "synthetic (seeded)", "config": describe(args.workload, w),
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def live_peaks(fc) -> dict:
    """Rates of the units that bound the kernels on this GPU, measured now by
    the library's probes (fc_probe_rate): L2 reads, shared-memory atomics,
    64-bit AND + popcount."""
    return {"l2_read_gbs_4mib": fc.fc_probe_rate(fc.FC_PROBE_L2_READ, 4 << 20) / 1e9,
            "l2_read_gbs_64mib": fc.fc_probe_rate(fc.FC_PROBE_L2_READ, 64 << 20) / 1e9,
            "smem_atomics_g_per_s": fc.fc_probe_rate(fc.FC_PROBE_SMEM_ATOMIC) / 1e9,
            "and_popc_g_words_per_s": fc.fc_probe_rate(fc.FC_PROBE_AND_POPC) / 1e9}


def roofline(name: str, ms: float, work: dict, pk: dict, resident_bytes: int, plan_sig: str) -> dict:
    """Roofline of the step's dominant kernel: the algorithmic work of one
    step over the step's device time, against the measured rate of the unit
    that bounds it (`pk`: probe rates measured on this GPU by this run, plus
    MEASURED_PEAKS.json's HBM and bf16 figures)."""
    sec = ms / 1e3
    hbm, bf16 = pk["hbm_gbs"], pk["bf16_tflops"]
    l2 = pk["l2_read_gbs_4mib"] if resident_bytes <= (8 << 20) else pk["l2_read_gbs_64mib"]
    traffic = measured_traffic(name, plan_sig)
    if name == "pairs":
        achieved = work["flops"] / sec / 1e12
        peak = bf16 * 2.0
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic,
                "peak_source": f"{pk['src']} bf16 burst x 2 (the nominal fp8/bf16 ratio; e4m3 operands)",
                "duration": "whole step (the GEMM and the table/MI extraction)"}
    if name in ("support", "splits", "assign"):
        achieved = work["popc_words"] / sec / 1e9
        peak = pk["and_popc_g_words_per_s"]
        r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G words/s", "frac": achieved / peak,
             "traffic": traffic,
             "peak_source": "measured by fc_probe_rate(FC_PROBE_AND_POPC) on this GPU: 64-bit AND + popcount + add",
             "work": "one 64-bit AND + popcount per word of every set counted "
                     + ("(the 2^k - 1 - k subsets of >= 2 items of each itemset; one-item subsets are the "
                        "marginals counted at load)" if name == "splits" else
                        "(the itemset and its k leave-one-out sets; for k = 2 those are single items, whose "
                        "counts are the marginals counted at load)" if name == "support"
                        else "(the AND of the conditions' state bitmaps)"),
             "duration": "whole step"}
        if resident_bytes > L2_BYTES:
            r["hbm"] = {"achieved": work["alg_bytes"] / sec / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": work["alg_bytes"] / sec / 1e9 / hbm,
                        "note": "algorithmic bytes (k bitmap rows per itemset) over the step; the range-major "
                                "order re-reads each bitmap slice from L2, not HBM"}
        return r
    if name in ("tiny", "random", "large", "scores"):
        achieved = work["atomics"] / sec / 1e9
        peak = pk["smem_atomics_g_per_s"]
        r = {"bound": "smem_atomic", "achieved": achieved, "peak": peak, "unit": "G atomics/s",
             "frac": achieved / peak, "traffic": traffic,
             "peak_source": "measured by fc_probe_rate(FC_PROBE_SMEM_ATOMIC) on this GPU: conflict-free "
                            "shared-memory atomicAdd, all lanes busy",
             "work": "one shared-memory atomic per instance of every query counted by a key strategy "
                     f"({work['keyed_queries']} of {work['queries']} queries)",
             "duration": "whole step",
             "l2": {"achieved": work["col_bytes"] / sec / 1e9, "peak": l2, "unit": "GB/s",
                    "frac": work["col_bytes"] / sec / 1e9 / l2,
                    "work": "k column values per instance of every keyed query, read from L2 at the "
                            "width the histogram keys read them (4 bits per value with the 4-bit columns)"},
             "effective_gbs": work["alg_bytes"] / sec / 1e9}
        if name == "scores":
            r["note"] = (f"the step also runs the bitmap launch of {work['queries'] - work['keyed_queries']} "
                         "queries; its time is in the denominator, its work is not")
        if name == "tiny":
            r["note"] = "launch- and latency-bound: 92 queries of 1,000 instances"
        if name == "large":
            r["note"] = ("tables beyond shared memory, counted window by window: every row is keyed once per "
                         "window and only the keys inside it are counted, so the launch is bound by the key "
                         "arithmetic (ALU), not by the atomics this fraction counts")
        return r
    # families, rules, append: byte-bound work
    achieved = work["alg_bytes"] / sec / 1e9
    if resident_bytes < L2_BYTES and name != "append":
        r = {"bound": "l2", "achieved": achieved, "peak": l2, "unit": "GB/s", "frac": achieved / l2,
             "traffic": traffic, "peak_source": "measured by fc_probe_rate(FC_PROBE_L2_READ) on this GPU",
             "duration": "whole step"}
        if name == "families":
            r["work"] = ("the columns of every variable set counted once, at the width the histogram keys "
                         "read them (4 bits per value with the 4-bit columns)")
        return r
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "peak_source": f"{pk['src']} hbm_gbs", "duration": "whole step"}


def setup_gpu(args, rank: int, world: int):
    import torch

    import paper_1804_04640_gb300 as fc

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    fc.load_library(build_if_missing=True)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    hbm, bf16, bf16_sus, src = peaks()
    pk = dict(live_peaks(fc), hbm_gbs=hbm, bf16_tflops=bf16, src=src)
    return torch, fc, dist, dev, barrier, pk


def set_options(fc, args, ctx):
    """Apply the --option KEY=VALUE settings to a freshly loaded context."""
    for kv in getattr(args, "option", None) or []:
        key, value = kv.split("=", 1)
        fc.fc_set_option(ctx, key, int(value))
    return ctx


def load_ctx(fc, args, D, arities):
    return set_options(fc, args, fc.fc_load(D, arities))


def measure(name: str, args, rank: int, world: int, torch, fc, dist, dev, barrier, pk,
            steps: int | None, cpu_seconds: float, per_query_n: int, clk, nvtx: bool = False):
    """One workload on this GPU: device-timed steps of its plan, the
    per-query launches (random), the host-buffer entry point end to end, the
    roofline and the CPU oracle baseline.  Returns the record (rank 0)."""
    w = make_workload(name, args.m, args.nq, rank, world)
    stream = torch.cuda.Stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    work = {}
    per_query = None
    extra = {}
    if name in ("tiny", "random", "large"):
        db, queries = w["db"], w["queries"]
        ctx = load_ctx(fc, args, db.D, db.arities)
        off, flat = fc.pack_lists(queries)
        if args.autotune:
            fc.fc_autotune_batch(ctx, off, flat)
        fc.fc_set_option(ctx, "strategy", args.strategy)
        plan = fc.fc_plan_count(ctx, off, flat)
        toff = fc.fc_plan_table_offsets(plan)
        outs = (torch.empty(int(toff[-1]), dtype=torch.int32, device="cuda"),)
        units = len(queries)
        strat = fc.fc_plan_strategies(plan)
        keyed = np.isin(strat, [fc.FC_STRAT_HIST, fc.FC_STRAT_WINDOW, fc.FC_STRAT_GATOMIC, fc.FC_STRAT_SORT])
        ks = np.array([len(q) for q in queries])
        work = {"alg_bytes": int(ks.sum()) * db.m + 4 * int(toff[-1]), "atomics": int(keyed.sum()) * db.m,
                "col_bytes": int(ks[keyed].sum()) * db.m * fc.fc_info(ctx, 6) // 8,
                "keyed_queries": int(keyed.sum()), "queries": units}
        pinned = torch.empty(int(toff[-1]), dtype=torch.int32).pin_memory()
        h2d = fc.fc_plan_size(plan, 5) + 4 * (len(off) + len(flat))
        d2h = 4 * int(toff[-1])
        # the step's inputs in page-locked host memory, as the caller would
        # hold them (numpy views of pinned tensors: no per-call conversion)
        pin_in = [torch.from_numpy(np.ascontiguousarray(a, dtype=t)).pin_memory()
                  for a, t in ((off, np.int32), (flat, np.int32), (toff, np.int64))]
        p_off, p_flat, p_toff = (t.numpy() for t in pin_in)

        def e2e_call():
            fc.fc_count_batch(ctx, p_off, p_flat, p_toff, out=pinned)

        if name == "random" and per_query_n > 0:
            per_plans, pq_outs = [], []
            for q in queries[:min(per_query_n, len(queries))]:
                o1, f1 = fc.pack_lists([q])
                p1 = fc.fc_plan_count(ctx, o1, f1)
                per_plans.append(p1)
                pq_outs.append(torch.empty(max(fc.fc_plan_size(p1, 0), 1), dtype=torch.int32, device="cuda"))
            per_query = (per_plans, pq_outs)
        strategies = np.bincount(strat, minlength=6).tolist()
    elif name == "scores":
        db = w["db"]
        ctx = load_ctx(fc, args, db.D, db.arities)
        po, pa = fc.pack_lists(w["parents"])
        if args.autotune:  # the counting work of a score query is the table over (parents..., child)
            fo, ff = fc.pack_lists([list(p) + [c] for p, c in zip(w["parents"], w["child"])])
            fc.fc_autotune_batch(ctx, fo, ff)
        fc.fc_set_option(ctx, "strategy", args.strategy)
        plan = fc.fc_plan_score(ctx, w["child"], po, pa, "bdeu", 1.0)
        outs = (torch.empty(len(w["child"]), dtype=torch.float32, device="cuda"),)
        units = len(w["child"])
        strat = fc.fc_plan_strategies(plan)
        keyed = np.isin(strat, [fc.FC_STRAT_HIST, fc.FC_STRAT_WINDOW, fc.FC_STRAT_GATOMIC, fc.FC_STRAT_SORT])
        ks = np.array([len(p) + 1 for p in w["parents"]])
        work = {"alg_bytes": int(ks.sum()) * db.m, "atomics": int(keyed.sum()) * db.m,
                "col_bytes": int(ks[keyed].sum()) * db.m * fc.fc_info(ctx, 6) // 8,
                "keyed_queries": int(keyed.sum()), "queries": units}
        pinned = torch.empty(units, dtype=torch.float32).pin_memory()
        h2d = fc.fc_plan_size(plan, 5) + 4 * (units + len(po) + len(pa))
        d2h = 4 * units

        def e2e_call():
            fc.fc_score_batch(ctx, w["child"], po, pa, "bdeu", 1.0, out=pinned)
        strategies = np.bincount(strat, minlength=6).tolist()
    elif name == "families":
        db = w["db"]
        ctx = load_ctx(fc, args, db.D, db.arities)
        fams = fc.family_list(w["vars"], w["max_parents"])
        po, pa = fc.pack_lists([f[1] for f in fams])
        if args.autotune:
            fo, ff = fc.pack_lists([list(f[1]) + [f[0]] for f in fams])
            fc.fc_autotune_batch(ctx, fo, ff)
        plan = fc.fc_plan_families(ctx, w["vars"], w["max_parents"], "bdeu", 1.0)
        units = fc.fc_plan_size(plan, 1)
        outs = (torch.empty(units, dtype=torch.float32, device="cuda"),)
        nv, dmax = len(w["vars"]), min(w["max_parents"], len(w["vars"]) - 1)
        import math
        # every variable set's columns, at the width the histogram keys read them
        work = {"alg_bytes": sum(math.comb(nv, sz) * sz for sz in range(1, dmax + 2)) * db.m
                * fc.fc_info(ctx, 6) // 8}
        pinned = torch.empty(units, dtype=torch.float32).pin_memory()
        h2d = fc.fc_plan_size(plan, 5)
        d2h = 4 * units
        # the same families with one table per family (no sharing of variable sets)
        per_family_plan = fc.fc_plan_score(ctx, [f[0] for f in fams], po, pa, "bdeu", 1.0)
        per_family_out = torch.empty(units, dtype=torch.float32, device="cuda")

        def e2e_call():
            fc.fc_score_families(ctx, w["vars"], w["max_parents"], "bdeu", 1.0, out=pinned)
        strategies = None
    elif name == "assign":
        db = w["db"]
        ctx = load_ctx(fc, args, db.D, db.arities)
        vo, vv = fc.pack_lists([q[0] for q in w["assign"]])
        _, ss = fc.pack_lists([q[1] for q in w["assign"]])
        plan = fc.fc_plan_assignments(ctx, vo, vv, ss)
        units = len(w["assign"])
        outs = (torch.empty(units, dtype=torch.int32, device="cuda"),)
        words = (db.m + 63) // 64
        work = {"alg_bytes": int(len(vv)) * words * 8, "popc_words": units * words}
        pinned = torch.empty(units, dtype=torch.int64).pin_memory()
        h2d = fc.fc_plan_size(plan, 5) + 4 * (len(vo) + 2 * len(vv))
        d2h = 4 * units

        def e2e_call():
            fc.fc_count_assignment_batch(ctx, vo, vv, ss, out=pinned)
        strategies = None
    elif name == "pairs":
        db = w["db"]
        ctx = load_ctx(fc, args, db.D, db.arities)
        plan = fc.fc_plan_pairs(ctx)
        outs = (torch.empty(fc.fc_plan_size(plan, 0), dtype=torch.int32, device="cuda"),
                torch.empty(fc.fc_plan_size(plan, 1), dtype=torch.float32, device="cuda"))
        units = fc.fc_plan_size(plan, 1)
        R = int(db.arities.sum())
        work = {"flops": R * (R + 1) // 2 * 2 * db.m}
        pin_t = torch.empty(outs[0].numel(), dtype=torch.int32).pin_memory()
        pin_m = torch.empty(outs[1].numel(), dtype=torch.float32).pin_memory()
        h2d = 0
        d2h = 4 * (outs[0].numel() + outs[1].numel())

        def e2e_call():
            fc.load_library().fc_pairs_all(ctx.ptr, fc._ptr(pin_t), fc._ptr(pin_m))
        strategies = None
    else:
        ctx = set_options(fc, args, fc.fc_load_bits(w["bits"], w["m"]))
        so, it = fc.pack_lists(w["sets"])
        splits = name == "splits"
        plan = fc.fc_plan_support_splits(ctx, so, it) if splits else fc.fc_plan_support(ctx, so, it)
        n_out = fc.fc_plan_size(plan, 3)
        outs = (torch.empty(len(w["sets"]), dtype=torch.int32, device="cuda"),
                torch.empty(n_out, dtype=torch.int32, device="cuda"),
                torch.empty(n_out, dtype=torch.float32, device="cuda"))
        units = len(w["sets"])
        words = (w["m"] + 63) // 64
        ks = np.diff(so).astype(np.int64)
        # sets counted per word: one-item sets are the load-time marginals,
        # so every subset of >= 2 items (splits), or the itemset and its k
        # leave-one-out sets when those have >= 2 items (supports)
        sets_per = (2 ** ks - 1 - ks) if splits else np.where(ks == 2, 1, ks + 1)
        work = {"alg_bytes": int(len(it)) * (w["m"] // 8), "popc_words": int(sets_per.sum()) * words}
        pins = tuple(torch.empty(o.numel(), dtype=o.dtype).pin_memory() for o in outs)
        h2d = fc.fc_plan_size(plan, 5)
        d2h = sum(4 * o.numel() for o in outs)

        def e2e_call():
            if splits:
                fc.fc_support_splits_batch(ctx, so, it, out=pins)
            else:
                fc.fc_support_batch(ctx, so, it, out=pins)
        strategies = None

    # bytes the step's kernels read from the database (columns or state bitmaps)
    if name in ("support", "splits"):
        resident_bytes = int(np.asarray(w["bits"]).nbytes)
    elif name == "assign":
        resident_bytes = int(w["db"].arities.sum()) * ((w["db"].m + 63) // 64) * 8
    else:
        resident_bytes = w["db"].n * w["db"].m

    def step():
        fc.fc_plan_run(plan, *outs, stream=stream)

    # ---- warm-up (also captures the graph); a step's time picks the count
    # of timed steps when the caller leaves it open (about 1 s of steps)
    t_warm = []
    for _ in range(args.warmup):
        flush.fill_(1)
        stream.wait_stream(torch.cuda.current_stream())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        t_warm.append(e0.elapsed_time(e1))
    fc.fc_sync(ctx, stream)
    if steps is None:
        cap = args.steps if args.steps is not None else 2000
        steps = int(max(3, min(cap, 1000.0 / max(min(t_warm), 1e-3))))

    # ---- timed region: K steps, L2 flushed between steps, events on the launch stream
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    barrier()
    if nvtx:  # names the timed region for profilers (ncu --nvtx --nvtx-include timed/)
        try:
            torch.cuda.nvtx.range_push("timed")
        except Exception:  # noqa: BLE001
            nvtx = False
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(i)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    barrier()
    if nvtx:
        torch.cuda.nvtx.range_pop()
    times = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    fc.fc_sync(ctx, stream)
    ms = float(np.mean(times))
    total_ms = float(np.sum(times))
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    # every rank answered its own `units` (its slice of the job's batch, or
    # its own problem): the job's throughput counts each once
    value = units * world * steps / (total_ms / 1e3)

    # ---- per-query launches (same kernel, one launch per query)
    if per_query is not None:
        plans, pouts = per_query
        for p1, o in zip(plans, pouts):      # warm-up / capture
            fc.fc_plan_run(p1, o, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for p1, o in zip(plans, pouts):
            fc.fc_plan_run(p1, o, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        pq_ms = e0.elapsed_time(e1)
        extra["per_query"] = {"value": len(plans) / (pq_ms / 1e3), "unit": "queries/s", "queries": len(plans),
                              "launches": len(plans)}
        extra["batched_over_per_query"] = units / (ms / 1e3) / extra["per_query"]["value"]

    # ---- families: the same families with one counted table each
    if name == "families":
        for _ in range(2):
            fc.fc_plan_run(per_family_plan, per_family_out, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(3, min(steps, 10))
        e0.record(stream)
        for _ in range(reps):
            fc.fc_plan_run(per_family_plan, per_family_out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        pf_ms = e0.elapsed_time(e1) / reps
        extra["per_family_tables"] = {"value": units / (pf_ms / 1e3), "unit": "families/s", "ms_per_step": pf_ms,
                                      "note": "one counted table per family (fc_plan_score)"}

    # ---- end to end through the host-buffer entry point
    for _ in range(3):
        e2e_call()
    e2e_t = []
    for _ in range(max(5, min(steps, 50, int(2000.0 / max(ms, 1e-3))))):  # about 2 s at most
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_call()
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = float(np.median(e2e_t))
    clk.stop()
    planner = "host"
    if name in ("tiny", "random", "large") and fc.fc_info(ctx, 7) == 1:
        # planned on the device: only the query lists and the caller's table
        # offsets are uploaded (the entropies stay on the device)
        planner = "device"
        h2d = 4 * (len(off) + len(flat)) + 8 * len(toff)

    plan_sig = "-"
    if strategies is not None:
        plan_sig = ",".join(f"{n}={c}" for n, c in zip(STRATEGY_NAMES, strategies) if c)
    roof = roofline(name, ms, work, pk, resident_bytes, plan_sig)
    rec = None
    if rank == 0:
        cores = os.cpu_count() or 1
        cpu = None
        if world == 1 and cpu_seconds > 0:
            rate, sample = oracle_rate(name, w, cpu_seconds, cores)
            cpu = {"value": rate, "unit": UNITS[name], "cores": cores, "kind": "oracle", "sample": sample}
        rec = {
            "metric": metric_of(name), "value": value, "unit": UNITS[name], "steps": steps,
            "ms_per_step": ms,
            "dtype": {"pairs": "e4m3 one-hot x f32 accumulate -> int32"}.get(name, "u8/int32"),
            "config": with_options(describe(name, w), args),
            "e2e": {"value": units / e2e_s, "unit": UNITS[name], "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "planner": planner},
            "gpu_launches": steps * fc.fc_plan_size(plan, 6),
            "roofline": roof, "cpu_baseline": cpu,
            "plan": {"kernels_per_step": fc.fc_plan_size(plan, 6), "signature": plan_sig,
                     "l2": "flushed between timed steps (256 MiB write)"},
        }
        if strategies is not None:
            rec["plan"]["strategies"] = dict(zip(STRATEGY_NAMES, strategies))
            rec["plan"]["cost_model_fs"] = {k: fc.fc_get_option(ctx, k) for k in
                                            ("bitmap_cost", "bitmap_chunk_cost", "small_cost", "small3_cost", "hist_cost_row",
                                             "hist_cost_var")}
        rec.update(extra)
    del plan, ctx
    return rec


def run_gpu(args, rank: int, world: int):
    torch, fc, dist, dev, barrier, pk = setup_gpu(args, rank, world)
    name = args.workload
    if name == "rules":
        return run_rules_gpu(args, rank, world, fc, torch, barrier, dist, dev, pk)
    if name == "append":
        return run_append_gpu(args, rank, world, fc, torch, barrier, dist, dev, pk)
    # clocks are sampled from before the warm-up to after the end-to-end leg
    with ClockSampler(dev) as clk:
        rec = measure(name, args, rank, world, torch, fc, dist, dev, barrier, pk, args.steps,
                      0.0 if args.no_cpu_baseline else args.cpu_seconds, args.per_query, clk, nvtx=True)
    line = None
    if rank == 0:
        line = {"metric": rec["metric"], "value": rec["value"], "unit": rec["unit"], "n_gpus": world,
                "steps": rec["steps"], "warmup": args.warmup, "ms_per_step": rec["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": rec["dtype"],
                "data": "synthetic (seeded random-DAG samples)", "config": rec["config"],
                "e2e": rec["e2e"], "gpu_launches": rec["gpu_launches"], "roofline": rec["roofline"],
                "cpu_baseline": rec["cpu_baseline"], "clocks": clk.summary(), "plan": rec["plan"],
                "probe_peaks": {k: v for k, v in pk.items() if k not in ("src",)}}
        for k in ("per_query", "batched_over_per_query", "per_family_tables"):
            if k in rec:
                line[k] = rec[k]
        if world > 1:
            line["sharding"] = ("each rank answers its own slice of one batch of n_gpus x the workload's "
                                "queries (shard.split_batch); the database is replicated, no exchange")
    # the other benchmark configurations, each with its own clocks (one GPU only)
    if args.all_configs and world == 1 and name == "random":
        nested = {}
        for other in NESTED:
            with ClockSampler(dev) as clk2:
                r2 = measure(other, argparse.Namespace(**dict(vars(args), m=None, nq=None)), rank, world, torch,
                             fc, dist, dev, barrier, pk, None,
                             0.0 if args.no_cpu_baseline else args.config_cpu_seconds, 0, clk2)
            r2["clocks"] = clk2.summary()
            nested[other] = r2
            torch.cuda.empty_cache()
        if line is not None:
            line["configs"] = nested
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return line


def run_rules_gpu(args, rank, world, fc, torch, barrier, dist, dev, pk):
    """One step = one whole fc_mine_rules call (host candidate generation,
    one counting launch per level, counts read back), timed with CUDA events
    around the synchronous call on an idle device."""
    name = "rules"
    w = make_workload(name, args.m, args.nq, rank, world)
    db = w["db"]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    ctx = load_ctx(fc, args, db.D, db.arities)
    clk = ClockSampler(dev).__enter__()
    for _ in range(args.warmup):
        r = fc.fc_mine_rules(ctx, *w["args"])
    torch.cuda.synchronize()
    units = r["candidates"]
    steps = args.steps if args.steps is not None else 50
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    dev_ns = []
    barrier()
    for i in range(steps):
        flush.fill_(i)
        torch.cuda.synchronize()
        starts[i].record()
        r = fc.fc_mine_rules(ctx, *w["args"])
        ends[i].record()
        dev_ns.append(r["device_ns"])
    barrier()
    times = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms = float(np.mean(times))
    total_ms = float(np.sum(times))
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = units * world * steps / (total_ms / 1e3)

    # end to end: load the database from host memory, mine, results on the host
    e2e_t = []
    for _ in range(max(3, min(steps, 10))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = load_ctx(fc, args, db.D, db.arities)
        r2 = fc.fc_mine_rules(c2, *w["args"])
        del c2
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = float(np.median(e2e_t))
    clk.stop()

    # dominant kernel: the per-level itemset count; algorithmic bytes = one
    # bitmap row of ceil(m/64) words per item of every candidate
    sizes = np.diff(r["set_off"])
    row_bytes = (db.m + 63) // 64 * 8
    dev_ms = float(np.median(dev_ns)) / 1e6
    line = None
    if rank == 0:
        cores = os.cpu_count() or 1
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            rate, sample = oracle_rate(name, w, args.cpu_seconds, cores)
            cpu = {"value": rate, "unit": UNITS[name], "cores": 1, "kind": "oracle", "sample": sample}
        alg_bytes = r["candidate_items"] * row_bytes
        line = {
            "metric": f"{name}: {UNITS[name]}", "value": value, "unit": UNITS[name], "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8/int32",
            "data": "synthetic (seeded random-DAG samples)",
            "config": with_options(describe(name, w), args),
            "plan": {"l2": "flushed between timed steps (256 MiB write)",
                     "frequent_itemsets": int(len(sizes)), "rules": int(len(r["rule_set"])),
                     "candidates": int(units), "levels": int(r["levels"]),
                     "max_itemset": int(sizes.max()) if len(sizes) else 0},
            "e2e": {"value": units / e2e_s, "unit": UNITS[name],
                    "h2d_bytes_per_step": int(db.n * db.m + r2["h2d_bytes"]),
                    "d2h_bytes_per_step": int(r2["d2h_bytes"])},
            "gpu_launches": steps * int(r["levels"]),
            "device_ms_per_step": dev_ms,
            "cpu_baseline": cpu, "clocks": clk.summary(),
        }
        if dev_ms > 0:
            achieved = alg_bytes / (dev_ms / 1e3) / 1e9
            l2 = pk["l2_read_gbs_64mib"]
            line["roofline"] = {
                "bound": "l2", "achieved": achieved, "peak": l2, "unit": "GB/s", "frac": achieved / l2,
                "traffic": None, "peak_source": "measured by fc_probe_rate(FC_PROBE_L2_READ) on this GPU",
                "note": (f"bytes/s of the counting launches (device time of the levels, {dev_ms:.3f} ms of "
                         f"{ms:.3f} ms per step); the {db.arities.sum() * row_bytes / 2**20:.0f} MiB of item "
                         "bitmaps stay in L2"),
                "duration": "sum of the per-level counting launches (CUDA events inside the library)"}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return line


def run_append_gpu(args, rank, world, fc, torch, barrier, dist, dev, pk):
    """One step = one fc_append of a block of instances that already sits in
    device memory (copy behind the old instances, state check, bitmap repack
    from the old m / 64, marginal update), timed with CUDA events around the
    synchronous call on an idle device; the context was reserved up front."""
    name = "append"
    w = make_workload(name, args.m, args.nq, rank, world)
    db, m0, B = w["db"], w["m0"], w["block"]
    D = np.ascontiguousarray(db.D)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    hbm, peak_src = pk["hbm_gbs"], pk["src"]
    # every step grows the database by a block: at most 50 steps (3.4 GB of D
    # and bitmaps per 50 blocks at n = 64), whatever --steps asks
    steps = min(args.steps, 50) if args.steps is not None else 50
    ctx = load_ctx(fc, args, D[:, :m0], db.arities)
    fc.fc_reserve(ctx, m0 + B * (args.warmup + steps + 1))
    block = torch.from_numpy(np.ascontiguousarray(D[:, m0:m0 + B])).cuda()
    clk = ClockSampler(dev).__enter__()
    for _ in range(args.warmup):
        fc.fc_append(ctx, block)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    barrier()
    for i in range(steps):
        flush.fill_(i)
        torch.cuda.synchronize()
        starts[i].record()
        fc.fc_append(ctx, block)
        ends[i].record()
    barrier()
    times = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms = float(np.mean(times))
    total_ms = float(np.sum(times))
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = B * world * steps / (total_ms / 1e3)
    # the grown context still answers like a single load (spot check)
    assert fc.fc_info(ctx, 1) == m0 + B * (args.warmup + steps)

    # end to end: the block comes from host memory (pinned) each step
    host_block = torch.from_numpy(np.ascontiguousarray(D[:, m0:m0 + B])).pin_memory()
    e2e_ctx = load_ctx(fc, args, D[:, :m0], db.arities)
    fc.fc_reserve(e2e_ctx, m0 + B * 12)
    e2e_t = []
    for _ in range(10):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fc.fc_append(e2e_ctx, host_block.numpy())
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = float(np.median(e2e_t[2:]))
    clk.stop()

    R = int(db.arities.sum())
    # algorithmic bytes per appended instance: read the new states and write
    # them behind D (2 n), read them once to check, pack and count them (n),
    # write R bits (R / 8)
    per_row = 3 * db.n + R / 8
    line = None
    if rank == 0:
        cores = os.cpu_count() or 1
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            rate, sample = oracle_rate(name, w, args.cpu_seconds, cores)
            cpu = {"value": rate, "unit": UNITS[name], "cores": 1, "kind": "oracle", "sample": sample}
        achieved = per_row * B / (ms / 1e3) / 1e9
        line = {
            "metric": f"{name}: {UNITS[name]}", "value": value, "unit": UNITS[name], "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (seeded random-DAG samples)",
            "config": with_options(describe(name, w), args),
            "plan": {"l2": "flushed between timed steps (256 MiB write)"},
            "e2e": {"value": B / e2e_s, "unit": UNITS[name], "h2d_bytes_per_step": int(db.n * B),
                    "d2h_bytes_per_step": int(8 * R + 4)},
            "gpu_launches": steps,  # the pack; the copy behind D is a driver memcpy
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": measured_traffic(name, "-"),
                         "peak_source": f"{peak_src} hbm_gbs",
                         "duration": "whole append call (copy, pack with the state check and marginal counts, "
                                     "host syncs); traffic is the pack's",
                         "note": f"algorithmic {per_row:.0f} B per appended instance"},
            "cpu_baseline": cpu, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return line


def measure_gemm_peaks():
    """Dense GEMM rates of the vendor library on this GPU (bf16, fp8 e4m3,
    int8), for the roofline denominators of the one-hot contraction; prints
    one JSON line.  Not part of any timed workload."""
    import torch
    res = {}
    n = 8192
    a16 = torch.randn(n, n, device="cuda", dtype=torch.bfloat16)
    b16 = torch.randn(n, n, device="cuda", dtype=torch.bfloat16)

    def rate(fn, flops, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return flops * reps / (e0.elapsed_time(e1) / 1e3) / 1e12

    res["bf16_tflops"] = rate(lambda: a16 @ b16, 2.0 * n ** 3)
    try:
        a8 = a16.to(torch.float8_e4m3fn)
        b8 = b16.to(torch.float8_e4m3fn).t().contiguous().t()
        one = torch.tensor(1.0, device="cuda")
        res["fp8_e4m3_tflops"] = rate(lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one,
                                                               out_dtype=torch.bfloat16), 2.0 * n ** 3)
    except Exception as e:  # noqa: BLE001
        res["fp8_e4m3_tflops"] = f"unavailable: {type(e).__name__}"
    try:
        ai = torch.randint(-8, 8, (n, n), device="cuda", dtype=torch.int8)
        bi = torch.randint(-8, 8, (n, n), device="cuda", dtype=torch.int8)
        res["int8_tops"] = rate(lambda: torch._int_mm(ai, bi), 2.0 * n ** 3)
    except Exception as e:  # noqa: BLE001
        res["int8_tops"] = f"unavailable: {type(e).__name__}"
    res["shape"] = f"{n} x {n} x {n}"
    res["library"] = "torch matmul / _scaled_mm / _int_mm (cuBLAS / cuBLASLt)"
    print(json.dumps(res), flush=True)


def measure_probe_peaks():
    """Print the probe rates (L2 reads, shared-memory atomics, AND + popcount)
    of this GPU as one JSON line."""
    import torch

    import paper_1804_04640_gb300 as fc
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    fc.load_library(build_if_missing=True)
    res = live_peaks(fc)
    for size in (1 << 20, 16 << 20, 32 << 20):
        res[f"l2_read_gbs_{size >> 20}mib"] = fc.fc_probe_rate(fc.FC_PROBE_L2_READ, size) / 1e9
    props = torch.cuda.get_device_properties(0)
    res["gpu"] = props.name
    res["sms"] = props.multi_processor_count
    res["how"] = "fc_probe_rate: best of 5 timed launches after one untimed, one full wave of CTAs"
    print(json.dumps(res), flush=True)


def relaunch_under_torchrun(n: int) -> int:
    """`bench.py --gpus N` started as one process: run it again as N ranks."""
    import socket
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: as many as take about a second, 3 to 2000; "
                         "given, exactly that many)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="random", choices=list(CONFIGS))
    ap.add_argument("--per-query", type=int, default=1000, help="queries timed with one launch each")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--config-cpu-seconds", type=float, default=4.0,
                    help="CPU oracle sample of each configuration nested under 'configs'")
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", dest="all_configs", action="store_false",
                    help="measure the headline workload only (by default a one-GPU run of the headline also "
                         "measures the other benchmark configurations and nests them under 'configs')")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip fc_autotune (strategy thresholds from the default cost model)")
    ap.add_argument("--option", action="append", default=[], metavar="KEY=VALUE",
                    help="fc_set_option on every context the bench loads (repeatable)")
    ap.add_argument("--strategy", type=int, default=-1, help="force one counting strategy (-1 = planner's choice)")
    ap.add_argument("--m", type=int, default=None, help="instances (default: the workload's own)")
    ap.add_argument("--nq", type=int, default=None, help="queries / itemsets (default: the workload's own)")
    ap.add_argument("--gemm-peaks", action="store_true",
                    help="only measure the vendor library's dense GEMM rates (bf16, fp8, int8) and exit")
    ap.add_argument("--peaks", action="store_true",
                    help="only measure the probe rates (L2 reads, shared-memory atomics, AND + popcount) and exit")
    args = ap.parse_args()
    if args.gemm_peaks:
        measure_gemm_peaks()
        return
    if args.peaks:
        measure_probe_peaks()
        return
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if "WORLD_SIZE" not in os.environ and args.gpus > 1:
        sys.exit(relaunch_under_torchrun(args.gpus))
    if world != args.gpus:
        sys.exit(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={world}; launch one rank per GPU")
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
