#!/usr/bin/env python3
"""Benchmark of the counting-query hot path on GB300.

Default workload ("random"): n = 40 categorical variables (arity 2-5),
m = 100,000 instances sampled from a random DAG, and a batch of 10,000 queries
of 2-6 variables drawn without replacement.  One step answers the whole batch
(every full contingency table) with one graph launch of the persistent count
kernel.  Printed as one JSON line:

  value      queries/s, device-resident inputs and outputs (max over ranks);
  e2e        the same through fc_count_batch with pinned host buffers
             (planning, host-to-device descriptors, kernel, device-to-host tables);
  per_query  the same queries issued as one launch each;
  roofline   the count kernel's effective bytes/s against the measured peak;
  cpu_baseline  the CPU oracle on a bounded sample, on this host's cores.

Other workloads (--workload tiny|scores|pairs|support) print their own line.
`--impl reference` times the CPU oracle on the same workload.
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

from workloads import (CONFIGS, config_database, random_queries, score_queries,  # noqa: E402
                       subset_queries, weighted_itemsets, zipf_item_probs, zipf_transaction_bitmaps)

L2_BYTES = 129 * 2**20


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), float(d.get("bf16_tflops_sustained", 0)), "measured"
    except Exception:
        return 6800.0, 1900.0, 1700.0, "fallback"


def measured_traffic(workload: str):
    """DRAM bytes per launch of the workload's dominant kernel from the committed
    ncu summary, or None when the kernel source changed since the capture."""
    import hashlib
    try:
        lines = open(os.path.join(ROOT, "profiles", "traffic.txt")).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        parts = ln.split()
        if len(parts) != 5 or ln.startswith("#") or parts[0] != workload:
            continue
        src = os.path.join(ROOT, "paper_1804_04640_gb300", "csrc", parts[2])
        try:
            sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        except OSError:
            return None
        return int(parts[4]) if sha == parts[3] else None
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
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
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ workloads

def make_workload(name: str, m: int | None = None, nq: int | None = None):
    """Seeded inputs of one workload (host arrays); m / nq shrink it (profiling)."""
    c = dict(CONFIGS[name])
    if m:
        c["m"] = m
    if nq:
        c["nq"] = nq
    if name in ("tiny", "random", "large"):
        db = config_database(name, c["m"])
        queries = subset_queries(db.n, (1, 2, 3)) if name == "tiny" else \
            random_queries(db.n, c["nq"], c["k"][0], c["k"][1], c["seed"])
        return {"db": db, "queries": queries}
    if name == "families":
        db = config_database("scores", c["m"])
        return {"db": db, "vars": list(range(c["nv"])), "max_parents": c["max_parents"]}
    if name == "rules":
        return {"db": config_database("scores", c["m"]), "args": (c["min_support"], c["min_confidence"],
                                                                  c["max_size"], False)}
    if name == "append":
        return {"db": config_database("scores", c["m"] + c["block"]), "m0": c["m"], "block": c["block"]}
    if name == "assign":
        db = config_database("random", c["m"])
        rng = np.random.default_rng(c["seed"])
        qs = []
        for _ in range(c["nq"]):
            k = int(rng.integers(c["k"][0], c["k"][1] + 1))
            vs = [int(x) for x in rng.choice(db.n, size=k, replace=False)]
            qs.append((vs, [int(rng.integers(0, db.arities[v])) for v in vs]))
        return {"db": db, "assign": qs}
    if name == "scores":
        db = config_database(name, c["m"])
        child, parents = score_queries(db.n, c["nq"], c["pa"][0], c["pa"][1], c["seed"])
        return {"db": db, "child": child, "parents": parents}
    if name == "pairs":
        return {"db": config_database(name, c["m"])}
    if name in ("support", "splits"):
        bits = zipf_transaction_bitmaps(c["n_items"], c["m"], c["zipf_s"], c["mean_len"], c["seed"])
        probs = zipf_item_probs(c["n_items"], c["zipf_s"], c["mean_len"])
        sets = weighted_itemsets(c["n_items"], c["nq"], c["k"][0], c["k"][1], probs, c["seed"])
        return {"bits": bits, "m": c["m"], "sets": sets}
    raise ValueError(name)


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
            import paper_1804_04640_gb300 as fcm
            orc = oracle.DB(w["db"].D, w["db"].arities)
            jobs = fcm.family_list(w["vars"], w["max_parents"])
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


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    w = make_workload(args.workload, args.m, args.nq)
    cores = os.cpu_count() or 1
    rate, sample = oracle_rate(args.workload, w, args.ref_seconds, cores)
    if args.workload in ("rules", "append"):
        cores = 1  # these oracle legs run on one thread
    steps = []
    for _ in range(args.warmup + args.steps):
        steps.append(oracle_rate(args.workload, w, max(0.5, args.ref_seconds / 4), cores)[0])
    value = statistics.median(steps[args.warmup:]) if args.steps else rate
    unit = UNITS[args.workload]
    line = {"impl": "reference", "metric": METRIC if args.workload == "random" else f"{args.workload}: {unit}",
            "value": value, "unit": unit, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64/f64",
            "data": "synthetic (seeded)", "config": describe(args.workload, w),
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def run_gpu(args, rank: int, world: int):
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

    name = args.workload
    if name == "rules":
        return run_rules_gpu(args, rank, world, fc, torch, barrier, dist, dev)
    if name == "append":
        return run_append_gpu(args, rank, world, fc, torch, barrier, dist, dev)
    w = make_workload(name, args.m, args.nq)
    stream = torch.cuda.Stream()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    hbm, bf16, bf16_sus, peak_src = peaks()

    # ---- set up the plan (device-resident inputs) and the e2e call
    per_query = None
    if name in ("tiny", "random", "large"):
        db, queries = w["db"], w["queries"]
        ctx = fc.fc_load(db.D, db.arities)
        off, flat = fc.pack_lists(queries)
        if args.autotune:
            fc.fc_autotune_batch(ctx, off, flat)
        fc.fc_set_option(ctx, "strategy", args.strategy)
        plan = fc.fc_plan_count(ctx, off, flat)
        toff = fc.fc_plan_table_offsets(plan)
        outs = (torch.empty(int(toff[-1]), dtype=torch.int32, device="cuda"),)
        units = len(queries)
        alg_bytes = sum(len(q) for q in queries) * db.m + 4 * int(toff[-1])
        pinned = torch.empty(int(toff[-1]), dtype=torch.int32).pin_memory()
        h2d = fc.fc_plan_size(plan, 5) + 4 * (len(off) + len(flat))
        d2h = 4 * int(toff[-1])

        def e2e_call():
            fc.fc_count_batch(ctx, off, flat, toff, out=pinned)

        if name == "random":
            nper = min(args.per_query, len(queries))
            per_plans = []
            pq_outs = []
            for q in queries[:nper]:
                o1, f1 = fc.pack_lists([q])
                p1 = fc.fc_plan_count(ctx, o1, f1)
                per_plans.append(p1)
                pq_outs.append(torch.empty(max(fc.fc_plan_size(p1, 0), 1), dtype=torch.int32, device="cuda"))
            per_query = (per_plans, pq_outs)
        strategies = np.bincount(fc.fc_plan_strategies(plan), minlength=6).tolist()
    elif name == "scores":
        db = w["db"]
        ctx = fc.fc_load(db.D, db.arities)
        po, pa = fc.pack_lists(w["parents"])
        if args.autotune:  # the counting work of a score query is the table over (parents..., child)
            fo, ff = fc.pack_lists([list(p) + [c] for p, c in zip(w["parents"], w["child"])])
            fc.fc_autotune_batch(ctx, fo, ff)
        fc.fc_set_option(ctx, "strategy", args.strategy)
        plan = fc.fc_plan_score(ctx, w["child"], po, pa, "bdeu", 1.0)
        outs = (torch.empty(len(w["child"]), dtype=torch.float32, device="cuda"),)
        units = len(w["child"])
        alg_bytes = (len(pa) + units) * db.m
        pinned = torch.empty(units, dtype=torch.float32).pin_memory()
        h2d = fc.fc_plan_size(plan, 5) + 4 * (units + len(po) + len(pa))
        d2h = 4 * units

        def e2e_call():
            fc.fc_score_batch(ctx, w["child"], po, pa, "bdeu", 1.0, out=pinned)
        strategies = np.bincount(fc.fc_plan_strategies(plan), minlength=6).tolist()
    elif name == "families":
        db = w["db"]
        ctx = fc.fc_load(db.D, db.arities)
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
        alg_bytes = sum(math.comb(nv, sz) * sz for sz in range(1, dmax + 2)) * db.m
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
        ctx = fc.fc_load(db.D, db.arities)
        vo, vv = fc.pack_lists([q[0] for q in w["assign"]])
        _, ss = fc.pack_lists([q[1] for q in w["assign"]])
        plan = fc.fc_plan_assignments(ctx, vo, vv, ss)
        units = len(w["assign"])
        outs = (torch.empty(units, dtype=torch.int32, device="cuda"),)
        alg_bytes = int(len(vv)) * ((db.m + 7) // 8)  # one state bitmap per condition
        pinned = torch.empty(units, dtype=torch.int64).pin_memory()
        h2d = fc.fc_plan_size(plan, 5) + 4 * (len(vo) + 2 * len(vv))
        d2h = 4 * units

        def e2e_call():
            fc.fc_count_assignment_batch(ctx, vo, vv, ss, out=pinned)
        strategies = None
    elif name == "pairs":
        db = w["db"]
        ctx = fc.fc_load(db.D, db.arities)
        plan = fc.fc_plan_pairs(ctx)
        outs = (torch.empty(fc.fc_plan_size(plan, 0), dtype=torch.int32, device="cuda"),
                torch.empty(fc.fc_plan_size(plan, 1), dtype=torch.float32, device="cuda"))
        units = fc.fc_plan_size(plan, 1)
        R = int(db.arities.sum())
        alg_flops = R * (R + 1) // 2 * 2 * db.m
        pin_t = torch.empty(outs[0].numel(), dtype=torch.int32).pin_memory()
        pin_m = torch.empty(outs[1].numel(), dtype=torch.float32).pin_memory()
        h2d = 0
        d2h = 4 * (outs[0].numel() + outs[1].numel())

        def e2e_call():
            fc.load_library().fc_pairs_all(ctx.ptr, fc._ptr(pin_t), fc._ptr(pin_m))
        strategies = None
    else:
        ctx = fc.fc_load_bits(w["bits"], w["m"])
        so, it = fc.pack_lists(w["sets"])
        splits = name == "splits"
        plan = fc.fc_plan_support_splits(ctx, so, it) if splits else fc.fc_plan_support(ctx, so, it)
        n_out = fc.fc_plan_size(plan, 3)
        outs = (torch.empty(len(w["sets"]), dtype=torch.int32, device="cuda"),
                torch.empty(n_out, dtype=torch.int32, device="cuda"),
                torch.empty(n_out, dtype=torch.float32, device="cuda"))
        units = len(w["sets"])
        alg_bytes = int(len(it)) * (w["m"] // 8)
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

    # ---- warm-up (also captures the graph)
    for _ in range(args.warmup):
        flush.fill_(1)
        stream.wait_stream(torch.cuda.current_stream())
        step()
    torch.cuda.synchronize()
    fc.fc_sync(ctx, stream)

    # ---- timed region: K steps, L2 flushed between steps, events on the launch stream
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    with ClockSampler(dev) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(i)
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        barrier()
        times = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    fc.fc_sync(ctx, stream)
    ms = float(np.mean(times))
    total_ms = float(np.sum(times))
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = units * world * args.steps / (total_ms / 1e3)

    # ---- per-query launches (same kernel, one launch per query)
    pq = None
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
        pq = {"value": len(plans) / (pq_ms / 1e3), "unit": "queries/s", "queries": len(plans),
              "launches": len(plans)}

    # ---- families: the same families with one counted table each
    pf = None
    if name == "families":
        for _ in range(2):
            fc.fc_plan_run(per_family_plan, per_family_out, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(3, min(args.steps, 10))
        e0.record(stream)
        for _ in range(reps):
            fc.fc_plan_run(per_family_plan, per_family_out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        pf_ms = e0.elapsed_time(e1) / reps
        pf = {"value": units / (pf_ms / 1e3), "unit": "families/s", "ms_per_step": pf_ms,
              "note": "one counted table per family (fc_plan_score)"}

    # ---- end to end through the host-buffer entry point
    for _ in range(2):
        e2e_call()
    e2e_t = []
    for _ in range(max(3, min(args.steps, 10))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_call()
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = float(np.median(e2e_t))

    # ---- roofline of the dominant kernel
    if name == "pairs":
        achieved = alg_flops / (ms / 1e3) / 1e12
        fp8_peak = bf16 * 2.0
        roof = {"bound": "tensor", "achieved": achieved, "peak": fp8_peak, "unit": "TFLOP/s",
                "frac": achieved / fp8_peak, "traffic": measured_traffic(name),
                "peak_source": f"{peak_src} bf16 burst x 2 (nominal fp8/bf16 ratio)"}
    else:
        achieved = alg_bytes / (ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": measured_traffic(name), "peak_source": f"{peak_src} hbm_gbs"}
        if resident_bytes < L2_BYTES:
            roof["note"] = (f"effective bytes/s: the {resident_bytes / 2**20:.0f} MiB the kernels read stay in "
                            "L2 after the first touch, so this is not an HBM fraction")
    roof["duration"] = (f"whole step ({fc.fc_plan_size(plan, 6)} kernels per step); the dominant kernel's "
                        "own share is in the committed launch list")

    line = None
    if rank == 0:
        cfg = describe(name, w)
        cfg["l2"] = "flushed between timed steps (256 MiB write)"
        if strategies is not None:
            cfg["strategies"] = dict(zip(["bitmap", "hist", "gatomic", "sort", "marginal", "window"], strategies))
            cfg["cost_model_fs"] = {k: fc.fc_get_option(ctx, k) for k in
                                    ("bitmap_cost", "bitmap_chunk_cost", "small_cost", "hist_cost_row", "hist_cost_var")}
        cores = os.cpu_count() or 1
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            rate, sample = oracle_rate(name, w, args.cpu_seconds, cores)
            cpu = {"value": rate, "unit": UNITS[name], "cores": cores, "kind": "oracle", "sample": sample}
        line = {
            "metric": METRIC if name == "random" else f"{name}: {UNITS[name]}",
            "value": value, "unit": UNITS[name], "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"pairs": "e4m3 one-hot x f32 accumulate -> int32"}.get(name, "u8/int32"),
            "data": "synthetic (seeded random-DAG samples)", "config": cfg,
            "e2e": {"value": units / e2e_s, "unit": UNITS[name], "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": args.steps * fc.fc_plan_size(plan, 6),
            "roofline": roof, "cpu_baseline": cpu, "clocks": clk.summary(),
        }
        if pq is not None:
            line["per_query"] = pq
            line["batched_over_per_query"] = value / world / pq["value"]
        if pf is not None:
            line["per_family_tables"] = pf
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return line


def run_rules_gpu(args, rank, world, fc, torch, barrier, dist, dev):
    """One step = one whole fc_mine_rules call (host candidate generation,
    one counting launch per level, counts read back), timed with CUDA events
    around the synchronous call on an idle device."""
    name = "rules"
    w = make_workload(name, args.m, args.nq)
    db = w["db"]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    hbm, _, _, peak_src = peaks()
    ctx = fc.fc_load(db.D, db.arities)
    for _ in range(args.warmup):
        r = fc.fc_mine_rules(ctx, *w["args"])
    torch.cuda.synchronize()
    units = r["candidates"]
    steps = min(args.steps, 50)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    dev_ns = []
    barrier()
    with ClockSampler(dev) as clk:
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
        c2 = fc.fc_load(db.D, db.arities)
        r2 = fc.fc_mine_rules(c2, *w["args"])
        del c2
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = float(np.median(e2e_t))

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
            "config": dict(describe(name, w), l2="flushed between timed steps (256 MiB write)",
                           frequent_itemsets=int(len(sizes)), rules=int(len(r["rule_set"])),
                           candidates=int(units), levels=int(r["levels"]),
                           max_itemset=int(sizes.max()) if len(sizes) else 0),
            "e2e": {"value": units / e2e_s, "unit": UNITS[name],
                    "h2d_bytes_per_step": int(db.n * db.m + r2["h2d_bytes"]),
                    "d2h_bytes_per_step": int(r2["d2h_bytes"])},
            "gpu_launches": steps * int(r["levels"]),
            "device_ms_per_step": dev_ms,
            "cpu_baseline": cpu, "clocks": clk.summary(),
        }
        if dev_ms > 0:
            achieved = alg_bytes / (dev_ms / 1e3) / 1e9
            line["roofline"] = {
                "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": None, "peak_source": f"{peak_src} hbm_gbs",
                "note": (f"effective bytes/s of the counting launches (device time of the levels, "
                         f"{dev_ms:.3f} ms of {ms:.3f} ms per step); the {db.arities.sum() * row_bytes / 2**20:.0f} "
                         "MiB of item bitmaps stay in L2, so this is not an HBM fraction"),
                "duration": "sum of the per-level counting launches (CUDA events inside the library)"}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return line


def run_append_gpu(args, rank, world, fc, torch, barrier, dist, dev):
    """One step = one fc_append of a block of instances that already sits in
    device memory (copy behind the old instances, state check, bitmap repack
    from the old m / 64, marginal update), timed with CUDA events around the
    synchronous call on an idle device; the context was reserved up front."""
    name = "append"
    w = make_workload(name, args.m, args.nq)
    db, m0, B = w["db"], w["m0"], w["block"]
    D = np.ascontiguousarray(db.D)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    hbm, _, _, peak_src = peaks()
    steps = min(args.steps, 50)
    ctx = fc.fc_load(D[:, :m0], db.arities)
    fc.fc_reserve(ctx, m0 + B * (args.warmup + steps + 1))
    block = torch.from_numpy(np.ascontiguousarray(D[:, m0:m0 + B])).cuda()
    for _ in range(args.warmup):
        fc.fc_append(ctx, block)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    barrier()
    with ClockSampler(dev) as clk:
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
    e2e_ctx = fc.fc_load(D[:, :m0], db.arities)
    fc.fc_reserve(e2e_ctx, m0 + B * 12)
    e2e_t = []
    for _ in range(10):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fc.fc_append(e2e_ctx, host_block.numpy())
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = float(np.median(e2e_t[2:]))

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
            "config": dict(describe(name, w), l2="flushed between timed steps (256 MiB write)"),
            "e2e": {"value": B / e2e_s, "unit": UNITS[name], "h2d_bytes_per_step": int(db.n * B),
                    "d2h_bytes_per_step": int(8 * R + 4)},
            "gpu_launches": steps,  # the pack; the copy behind D is a driver memcpy
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": measured_traffic(name),
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="random", choices=list(CONFIGS))
    ap.add_argument("--per-query", type=int, default=1000, help="queries timed with one launch each")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip fc_autotune (strategy thresholds from the default cost model)")
    ap.add_argument("--strategy", type=int, default=-1, help="force one counting strategy (-1 = planner's choice)")
    ap.add_argument("--m", type=int, default=None, help="instances (default: the workload's own)")
    ap.add_argument("--nq", type=int, default=None, help="queries / itemsets (default: the workload's own)")
    ap.add_argument("--gemm-peaks", action="store_true",
                    help="only measure the vendor library's dense GEMM rates (bf16, fp8, int8) and exit")
    args = ap.parse_args()
    if args.gemm_peaks:
        measure_gemm_peaks()
        return
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
