"""Python binding of libfc (include/fc.h): exact counting queries on a GB300.

The functions keep the names of the C ABI and only marshal arguments: numpy
arrays (or CPU torch tensors, e.g. pinned buffers) become host pointers, CUDA
torch tensors become device pointers.  Every computation runs in the CUDA
kernels of ``libfc.so``; there is no CPU fallback.  If the library has not
been built, or no CUDA device is usable, calls raise ``FcError``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

FC_OK, FC_ERR_ARG, FC_ERR_RANGE, FC_ERR_SIZE, FC_ERR_OOM, FC_ERR_CUDA, FC_ERR_TIMEOUT, FC_ERR_STATE = (
    0, -1, -2, -3, -4, -5, -6, -7)
FC_COL_MAJOR, FC_ROW_MAJOR = 0, 1
FC_HOST, FC_DEVICE = 0, 1
FC_LL, FC_MDL, FC_BDEU, FC_MI = 0, 1, 2, 3
(FC_STRAT_AUTO, FC_STRAT_BITMAP, FC_STRAT_HIST, FC_STRAT_GATOMIC, FC_STRAT_SORT, FC_STRAT_MARGINAL,
 FC_STRAT_WINDOW) = -1, 0, 1, 2, 3, 4, 5
SCORE_KINDS = {"ll": FC_LL, "mdl": FC_MDL, "bdeu": FC_BDEU, "mi": FC_MI}

# every entry point declared in include/fc.h
EXPORTS = (
    "fc_load", "fc_load_bits", "fc_free", "fc_info", "fc_marginals", "fc_count",
    "fc_count_assignment", "fc_count_batch", "fc_score_batch", "fc_pairs_all", "fc_pairs_cells",
    "fc_support_batch", "fc_plan_count", "fc_plan_score", "fc_plan_support", "fc_plan_pairs",
    "fc_plan_size", "fc_plan_table_offsets", "fc_plan_strategies", "fc_plan_run", "fc_plan_free",
    "fc_sync", "fc_set_option", "fc_get_option", "fc_autotune", "fc_last_error",
    "fc_selftest_wait_timeout", "fc_count_sorted_noalloc", "fc_autotune_batch",
    "fc_count_assignment_batch", "fc_plan_assignments", "fc_families_count", "fc_score_families",
    "fc_plan_families", "fc_mine_rules", "fc_rules_size", "fc_rules_itemsets", "fc_rules_list",
    "fc_rules_free", "fc_append", "fc_append_bits", "fc_reserve", "fc_support_splits_batch",
    "fc_plan_support_splits", "fc_probe_rate",
)


class FcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libfc error {code}: {msg}")
        self.code = code


_lib = None
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f32p = ctypes.POINTER(ctypes.c_float)
_vp = ctypes.c_void_p


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = False):
    """Load libfc.so (optionally compiling it first) and declare its symbols."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise FcError(FC_ERR_STATE, f"{path} is missing: build it with __graft_entry__.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    sig = {
        "fc_load": (ctypes.c_int, [ctypes.POINTER(_vp), _vp, ctypes.c_int32, ctypes.c_int64, _i32p,
                                   ctypes.c_int32, ctypes.c_int32]),
        "fc_load_bits": (ctypes.c_int, [ctypes.POINTER(_vp), _vp, ctypes.c_int32, ctypes.c_int64,
                                        ctypes.c_int32]),
        "fc_free": (None, [_vp]),
        "fc_info": (ctypes.c_int64, [_vp, ctypes.c_int32]),
        "fc_marginals": (ctypes.c_int, [_vp, _i64p]),
        "fc_count": (ctypes.c_int, [_vp, _i32p, ctypes.c_int32, _vp]),
        "fc_count_assignment": (ctypes.c_int, [_vp, _i32p, _i32p, ctypes.c_int32, _i64p]),
        "fc_count_batch": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, _i32p, _i64p, _vp]),
        "fc_score_batch": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, _i32p, _i32p, ctypes.c_int32,
                                          ctypes.c_double, _vp]),
        "fc_pairs_all": (ctypes.c_int, [_vp, _vp, _vp]),
        "fc_pairs_cells": (ctypes.c_int64, [_vp]),
        "fc_support_batch": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, _i32p, _vp, _vp, _vp]),
        "fc_plan_count": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, _i32p, _i64p, ctypes.POINTER(_vp)]),
        "fc_plan_score": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, _i32p, _i32p, ctypes.c_int32,
                                         ctypes.c_double, ctypes.POINTER(_vp)]),
        "fc_plan_support": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, _i32p, ctypes.POINTER(_vp)]),
        "fc_plan_pairs": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
        "fc_probe_rate": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), _vp]),
        "fc_plan_size": (ctypes.c_int64, [_vp, ctypes.c_int32]),
        "fc_plan_table_offsets": (ctypes.c_int, [_vp, _i64p]),
        "fc_plan_strategies": (ctypes.c_int, [_vp, _i32p]),
        "fc_plan_run": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
        "fc_plan_free": (None, [_vp]),
        "fc_sync": (ctypes.c_int, [_vp, _vp]),
        "fc_set_option": (ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.c_int64]),
        "fc_get_option": (ctypes.c_int64, [_vp, ctypes.c_char_p]),
        "fc_autotune": (ctypes.c_int, [_vp, ctypes.c_int32]),
        "fc_autotune_batch": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, _i32p]),
        "fc_families_count": (ctypes.c_int64, [ctypes.c_int32, ctypes.c_int32]),
        "fc_score_families": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_double, _vp]),
        "fc_plan_families": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_double, ctypes.POINTER(_vp)]),
        "fc_count_assignment_batch": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, _i32p, _i32p, _i64p]),
        "fc_plan_assignments": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, _i32p, _i32p, ctypes.POINTER(_vp)]),
        "fc_support_splits_batch": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, _i32p, _vp, _vp, _vp]),
        "fc_plan_support_splits": (ctypes.c_int, [_vp, ctypes.c_int32, _i32p, _i32p, ctypes.POINTER(_vp)]),
        "fc_mine_rules": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(_vp)]),
        "fc_rules_size": (ctypes.c_int64, [_vp, ctypes.c_int32]),
        "fc_rules_itemsets": (ctypes.c_int, [_vp, _i32p, _i32p, _i64p]),
        "fc_rules_list": (ctypes.c_int, [_vp, _i64p, ctypes.POINTER(ctypes.c_uint32), _f32p]),
        "fc_rules_free": (None, [_vp]),
        "fc_append": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]),
        "fc_append_bits": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_int32]),
        "fc_reserve": (ctypes.c_int, [_vp, ctypes.c_int64]),
        "fc_last_error": (ctypes.c_char_p, []),
        "fc_selftest_wait_timeout": (ctypes.c_int, [_vp, ctypes.c_int64]),
        "fc_count_sorted_noalloc": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _i32p,
                                                   _i32p, ctypes.c_int32, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != FC_OK:
        raise FcError(rc, _lib.fc_last_error().decode())


# ----------------------------------------------------------- marshalling

def _host(a, dtype):
    a = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    return a


def _ptr(a, ctype=None):
    """Pointer of a numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        p = a.data_ptr()
    else:
        p = a.ctypes.data
    return ctypes.cast(p, ctype) if ctype is not None else ctypes.c_void_p(p)


def _is_cuda(a) -> bool:
    return bool(getattr(a, "is_cuda", False))


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def pack_lists(lists):
    """[[...], ...] -> (offsets int32 (len+1), flat int32)."""
    off = np.zeros(len(lists) + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(x) for x in lists], dtype=np.int64)
    flat = np.fromiter((v for x in lists for v in x), dtype=np.int32, count=int(off[-1]))
    return off, flat


class Handle:
    """Owns a fc_ctx* or fc_plan* and frees it once."""

    def __init__(self, ptr, free, parent=None):
        self.ptr = ptr
        self._free = free
        self.parent = parent

    def close(self):
        if self.ptr:
            self._free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ entry points

def fc_load(D, arities, layout: int = FC_COL_MAJOR) -> Handle:
    """Load a uint8 database (numpy / CPU tensor, or CUDA tensor) onto the GPU."""
    lib = load_library()
    ar = _host(arities, np.int32)
    if _is_cuda(D):
        where, d = FC_DEVICE, D
    else:
        where, d = FC_HOST, _host(D, np.uint8)
    n, m = (d.shape[0], d.shape[1]) if layout == FC_COL_MAJOR else (d.shape[1], d.shape[0])
    out = _vp()
    _check(lib.fc_load(ctypes.byref(out), _ptr(d), int(n), int(m), _ptr(ar, _i32p), layout, where))
    h = Handle(out, lib.fc_free)
    h.arities = ar.astype(np.int64)
    return h


def fc_load_bits(bitmaps, m: int) -> Handle:
    lib = load_library()
    if _is_cuda(bitmaps):
        where, b = FC_DEVICE, bitmaps
    else:
        where, b = FC_HOST, _host(bitmaps, np.uint64)
    out = _vp()
    _check(lib.fc_load_bits(ctypes.byref(out), _ptr(b), int(b.shape[0]), int(m), where))
    h = Handle(out, lib.fc_free)
    h.arities = np.ones(int(b.shape[0]), dtype=np.int64)
    return h


def fc_append(ctx: Handle, D, layout: int = FC_COL_MAJOR):
    """Append instances (same forms as fc_load's D) to a categorical context."""
    lib = load_library()
    if _is_cuda(D):
        where, d = FC_DEVICE, D
    else:
        where, d = FC_HOST, _host(D, np.uint8)
    m_new = d.shape[1] if layout == FC_COL_MAJOR else d.shape[0]
    _check(lib.fc_append(ctx.ptr, _ptr(d), int(m_new), layout, where))


def fc_append_bits(ctx: Handle, bitmaps, m_new: int):
    """Append m_new transactions (n_items x ceil(m_new/64) uint64 bitmaps)."""
    lib = load_library()
    if _is_cuda(bitmaps):
        where, b = FC_DEVICE, bitmaps
    else:
        where, b = FC_HOST, _host(bitmaps, np.uint64)
    _check(lib.fc_append_bits(ctx.ptr, _ptr(b), int(m_new), where))


def fc_reserve(ctx: Handle, m_total: int):
    _check(load_library().fc_reserve(ctx.ptr, int(m_total)))


def fc_free(ctx: Handle):
    ctx.close()


def fc_info(ctx: Handle, key: int) -> int:
    return int(load_library().fc_info(ctx.ptr, key))


def fc_marginals(ctx: Handle) -> np.ndarray:
    out = np.zeros(fc_info(ctx, 2), dtype=np.int64)
    _check(load_library().fc_marginals(ctx.ptr, _ptr(out, _i64p)))
    return out


def fc_count(ctx: Handle, vars_) -> np.ndarray:
    lib = load_library()
    v = _host(vars_, np.int32)
    ar = fc_arities(ctx)
    cells = 1
    for x in v:
        cells *= int(ar[x]) if 0 <= x < len(ar) else 1
    # an oversized table is rejected by the library before anything is written
    out = np.zeros(cells if 0 < cells < 2**31 else 1, dtype=np.int32)
    _check(lib.fc_count(ctx.ptr, _ptr(v, _i32p), len(v), _ptr(out)))
    return out


def fc_count_assignment(ctx: Handle, vars_, states) -> int:
    lib = load_library()
    v, s = _host(vars_, np.int32), _host(states, np.int32)
    out = ctypes.c_int64(0)
    _check(lib.fc_count_assignment(ctx.ptr, _ptr(v, _i32p), _ptr(s, _i32p), len(v), ctypes.byref(out)))
    return int(out.value)


def fc_count_assignment_batch(ctx: Handle, var_off, vars_, states, out=None):
    """int64 count of each assignment (vars[t] = states[t] over each query's span)."""
    lib = load_library()
    vo, vv, st = _host(var_off, np.int32), _host(vars_, np.int32), _host(states, np.int32)
    nq = len(vo) - 1
    if out is None:
        out = np.zeros(max(nq, 1), dtype=np.int64)
    _check(lib.fc_count_assignment_batch(ctx.ptr, nq, _ptr(vo, _i32p), _ptr(vv, _i32p), _ptr(st, _i32p),
                                         _ptr(out, _i64p)))
    return out[:nq] if len(out) > nq else out


def fc_plan_assignments(ctx: Handle, var_off, vars_, states) -> Handle:
    lib = load_library()
    vo, vv, st = _host(var_off, np.int32), _host(vars_, np.int32), _host(states, np.int32)
    out = _vp()
    _check(lib.fc_plan_assignments(ctx.ptr, len(vo) - 1, _ptr(vo, _i32p), _ptr(vv, _i32p), _ptr(st, _i32p),
                                   ctypes.byref(out)))
    return Handle(out, lib.fc_plan_free, ctx)


def _table_offsets(ar, vo, vv) -> np.ndarray:
    """Dense table offsets (cells = product of arities per query, last fastest)."""
    nq = len(vo) - 1
    to = np.zeros(nq + 1, dtype=np.int64)
    if nq == 0:
        return to
    ar = np.asarray(ar, dtype=np.float64)
    vo = np.asarray(vo, dtype=np.int64)
    k = np.diff(vo)
    cells = np.ones(nq, dtype=np.float64)
    nz = k > 0
    if nz.any() and len(vv) >= vo[-1] and (k >= 0).all():
        # out-of-range ids count as arity 1 here; the library rejects them.
        # Segments start only at non-empty lists: an empty list's start is
        # the next list's, and each segment ends where the next one starts.
        ids = np.asarray(vv, dtype=np.int64)[:vo[-1]]
        ids = np.where((ids >= 0) & (ids < len(ar)), ids, len(ar))
        cells[nz] = np.multiply.reduceat(np.append(ar, 1.0)[ids], vo[:-1][nz])
    # tables past 2^31 cells are refused by the library (FC_ERR_SIZE); clamp
    # them so the offsets stay representable
    to[1:] = np.cumsum(np.minimum(cells, 2.0 ** 40).astype(np.int64))
    return to


def fc_count_batch(ctx: Handle, var_off, vars_, table_off=None, out=None):
    """Tables of a batch; returns (tables int32, table_off int64)."""
    lib = load_library()
    vo, vv = _host(var_off, np.int32), _host(vars_, np.int32)
    nq = len(vo) - 1
    if table_off is None:
        to = _table_offsets(fc_arities(ctx), vo, vv)
    else:
        to = _host(table_off, np.int64)
    if out is None:
        out = np.zeros(max(int(to[-1]), 1), dtype=np.int32)
    _check(lib.fc_count_batch(ctx.ptr, nq, _ptr(vo, _i32p), _ptr(vv, _i32p), _ptr(to, _i64p), _ptr(out)))
    return out, to


def fc_score_batch(ctx: Handle, child, par_off, parents, kind, ess: float = 1.0, out=None):
    lib = load_library()
    ch, po, pa = _host(child, np.int32), _host(par_off, np.int32), _host(parents, np.int32)
    kind = SCORE_KINDS.get(kind, kind)
    if out is None:
        out = np.zeros(max(len(ch), 1), dtype=np.float32)
    _check(lib.fc_score_batch(ctx.ptr, len(ch), _ptr(ch, _i32p), _ptr(po, _i32p), _ptr(pa, _i32p),
                              int(kind), float(ess), _ptr(out)))
    return out


def fc_families_count(nv: int, max_parents: int) -> int:
    return int(load_library().fc_families_count(int(nv), int(max_parents)))


def fc_score_families(ctx: Handle, vars_, max_parents: int, kind, ess: float = 1.0, out=None):
    """Scores of every (child, parent set) family over vars (layout in include/fc.h)."""
    lib = load_library()
    v = _host(vars_, np.int32)
    kind = SCORE_KINDS.get(kind, kind)
    if out is None:
        out = np.zeros(max(fc_families_count(len(v), max_parents), 1), dtype=np.float32)
    _check(lib.fc_score_families(ctx.ptr, len(v), _ptr(v, _i32p), int(max_parents), int(kind), float(ess),
                                 _ptr(out)))
    return out


def fc_plan_families(ctx: Handle, vars_, max_parents: int, kind, ess: float = 1.0) -> Handle:
    lib = load_library()
    v = _host(vars_, np.int32)
    kind = SCORE_KINDS.get(kind, kind)
    out = _vp()
    _check(lib.fc_plan_families(ctx.ptr, len(v), _ptr(v, _i32p), int(max_parents), int(kind), float(ess),
                                ctypes.byref(out)))
    return Handle(out, lib.fc_plan_free, ctx)


def family_list(vars_, max_parents: int):
    """(child, parents) of every family in the order fc_score_families writes them."""
    import itertools
    vs = [int(x) for x in vars_]
    nv = len(vs)
    d = min(max_parents, nv - 1)
    out = []
    for c in range(nv):
        others = [vs[i] for i in range(nv) if i != c]
        for s in range(d + 1):
            for comb in itertools.combinations(range(nv - 1), s):
                out.append((vs[c], [others[i] for i in comb]))
    return out


def fc_mine_rules(ctx: Handle, min_support: float, min_confidence: float, max_size: int,
                  all_splits: bool = False):
    """Bottom-up rule mining (layout in include/fc.h).

    Returns a dict: ``set_off``/``items``/``support`` (frequent itemsets, CSR),
    ``rule_set``/``antecedent``/``confidence`` (rules), and the number of
    ``candidates`` and ``levels`` counted on the device.
    """
    lib = load_library()
    h = _vp()
    _check(lib.fc_mine_rules(ctx.ptr, float(min_support), float(min_confidence), int(max_size),
                             int(bool(all_splits)), ctypes.byref(h)))
    try:
        ns, ni, nr = (int(lib.fc_rules_size(h, k)) for k in range(3))
        so = np.zeros(ns + 1, dtype=np.int32)
        it = np.zeros(max(ni, 1), dtype=np.int32)
        sp = np.zeros(max(ns, 1), dtype=np.int64)
        _check(lib.fc_rules_itemsets(h, _ptr(so, _i32p), _ptr(it, _i32p), _ptr(sp, _i64p)))
        rs = np.zeros(max(nr, 1), dtype=np.int64)
        ra = np.zeros(max(nr, 1), dtype=np.uint32)
        rc = np.zeros(max(nr, 1), dtype=np.float32)
        _check(lib.fc_rules_list(h, _ptr(rs, _i64p), ra.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                 _ptr(rc, _f32p)))
        return {"set_off": so, "items": it[:ni], "support": sp[:ns], "rule_set": rs[:nr],
                "antecedent": ra[:nr], "confidence": rc[:nr],
                "candidates": int(lib.fc_rules_size(h, 3)), "levels": int(lib.fc_rules_size(h, 4)),
                "h2d_bytes": int(lib.fc_rules_size(h, 5)), "d2h_bytes": int(lib.fc_rules_size(h, 6)),
                "device_ns": int(lib.fc_rules_size(h, 7)), "candidate_items": int(lib.fc_rules_size(h, 8))}
    finally:
        lib.fc_rules_free(h)


def fc_pairs_cells(ctx: Handle) -> int:
    return int(load_library().fc_pairs_cells(ctx.ptr))


def fc_pairs_all(ctx: Handle, tables: bool = True, mi: bool = True):
    lib = load_library()
    n = fc_info(ctx, 0)
    t = np.zeros(max(fc_pairs_cells(ctx), 1), dtype=np.int32) if tables else None
    m = np.zeros(max(n * (n - 1) // 2, 1), dtype=np.float32) if mi else None
    _check(lib.fc_pairs_all(ctx.ptr, _ptr(t), _ptr(m)))
    return t, m


def fc_support_batch(ctx: Handle, set_off, items, out=None):
    """(support, sub_support, confidence) of a batch of itemsets."""
    lib = load_library()
    so, it = _host(set_off, np.int32), _host(items, np.int32)
    nq = len(so) - 1
    if out is None:
        out = (np.zeros(max(nq, 1), dtype=np.int32), np.zeros(max(len(it), 1), dtype=np.int32),
               np.zeros(max(len(it), 1), dtype=np.float32))
    s, sub, conf = out
    _check(lib.fc_support_batch(ctx.ptr, nq, _ptr(so, _i32p), _ptr(it, _i32p), _ptr(s), _ptr(sub), _ptr(conf)))
    return s, sub, conf


def split_offsets(set_off) -> np.ndarray:
    """Start of each itemset's 2^k - 2 split entries (nq + 1 int64)."""
    so = np.asarray(set_off, dtype=np.int64)
    k = np.diff(so)
    n = np.where(k >= 2, (np.int64(1) << np.minimum(k, 62)) - 2, 0)
    return np.concatenate([[0], np.cumsum(n)]).astype(np.int64)


def fc_support_splits_batch(ctx: Handle, set_off, items, out=None):
    """(support, sub_support, confidence) over every antecedent split."""
    lib = load_library()
    so, it = _host(set_off, np.int32), _host(items, np.int32)
    nq = len(so) - 1
    ns = int(split_offsets(so)[-1])
    if out is None:
        out = (np.zeros(max(nq, 1), dtype=np.int32), np.zeros(max(ns, 1), dtype=np.int32),
               np.zeros(max(ns, 1), dtype=np.float32))
    s, sub, conf = out
    _check(lib.fc_support_splits_batch(ctx.ptr, nq, _ptr(so, _i32p), _ptr(it, _i32p), _ptr(s), _ptr(sub),
                                       _ptr(conf)))
    return s, sub, conf


def fc_plan_support_splits(ctx: Handle, set_off, items) -> Handle:
    lib = load_library()
    so, it = _host(set_off, np.int32), _host(items, np.int32)
    out = _vp()
    _check(lib.fc_plan_support_splits(ctx.ptr, len(so) - 1, _ptr(so, _i32p), _ptr(it, _i32p),
                                      ctypes.byref(out)))
    return Handle(out, lib.fc_plan_free, ctx)


def fc_plan_count(ctx: Handle, var_off, vars_, table_off=None) -> Handle:
    lib = load_library()
    vo, vv = _host(var_off, np.int32), _host(vars_, np.int32)
    to = None if table_off is None else _host(table_off, np.int64)
    out = _vp()
    _check(lib.fc_plan_count(ctx.ptr, len(vo) - 1, _ptr(vo, _i32p), _ptr(vv, _i32p), _ptr(to, _i64p),
                             ctypes.byref(out)))
    return Handle(out, lib.fc_plan_free, ctx)


def fc_plan_score(ctx: Handle, child, par_off, parents, kind, ess: float = 1.0) -> Handle:
    lib = load_library()
    ch, po, pa = _host(child, np.int32), _host(par_off, np.int32), _host(parents, np.int32)
    kind = SCORE_KINDS.get(kind, kind)
    out = _vp()
    _check(lib.fc_plan_score(ctx.ptr, len(ch), _ptr(ch, _i32p), _ptr(po, _i32p), _ptr(pa, _i32p), int(kind),
                             float(ess), ctypes.byref(out)))
    return Handle(out, lib.fc_plan_free, ctx)


def fc_plan_support(ctx: Handle, set_off, items) -> Handle:
    lib = load_library()
    so, it = _host(set_off, np.int32), _host(items, np.int32)
    out = _vp()
    _check(lib.fc_plan_support(ctx.ptr, len(so) - 1, _ptr(so, _i32p), _ptr(it, _i32p), ctypes.byref(out)))
    return Handle(out, lib.fc_plan_free, ctx)


def fc_plan_pairs(ctx: Handle) -> Handle:
    lib = load_library()
    out = _vp()
    _check(lib.fc_plan_pairs(ctx.ptr, ctypes.byref(out)))
    return Handle(out, lib.fc_plan_free, ctx)


def fc_plan_size(plan: Handle, key: int) -> int:
    return int(load_library().fc_plan_size(plan.ptr, key))


def fc_plan_table_offsets(plan: Handle) -> np.ndarray:
    out = np.zeros(fc_plan_size(plan, 4) + 1, dtype=np.int64)
    _check(load_library().fc_plan_table_offsets(plan.ptr, _ptr(out, _i64p)))
    return out


def fc_plan_strategies(plan: Handle) -> np.ndarray:
    out = np.zeros(max(fc_plan_size(plan, 4), 1), dtype=np.int32)
    _check(load_library().fc_plan_strategies(plan.ptr, _ptr(out, _i32p)))
    return out[: fc_plan_size(plan, 4)]


def fc_plan_run(plan: Handle, out0=None, out1=None, out2=None, stream=None):
    """Run a plan; outputs are CUDA tensors (device pointers)."""
    for o in (out0, out1, out2):
        if o is not None and not _is_cuda(o):
            raise FcError(FC_ERR_ARG, "fc_plan_run outputs must be CUDA tensors")
    _check(load_library().fc_plan_run(plan.ptr, _ptr(out0), _ptr(out1), _ptr(out2), _stream_ptr(stream)))


def fc_plan_free(plan: Handle):
    plan.close()


def fc_sync(ctx: Handle, stream=None):
    _check(load_library().fc_sync(ctx.ptr, _stream_ptr(stream)))


def fc_set_option(ctx: Handle, key: str, value: int):
    _check(load_library().fc_set_option(ctx.ptr, key.encode(), int(value)))


def fc_get_option(ctx: Handle, key: str) -> int:
    return int(load_library().fc_get_option(ctx.ptr, key.encode()))


def fc_autotune(ctx: Handle, budget_ms: int = 0):
    _check(load_library().fc_autotune(ctx.ptr, int(budget_ms)))


def fc_autotune_batch(ctx: Handle, var_off, vars_):
    vo, vv = _host(var_off, np.int32), _host(vars_, np.int32)
    _check(load_library().fc_autotune_batch(ctx.ptr, len(vo) - 1, _ptr(vo, _i32p), _ptr(vv, _i32p)))


def fc_last_error() -> str:
    return load_library().fc_last_error().decode()


def fc_selftest_wait_timeout(ctx: Handle, wait_limit: int) -> int:
    """Status of a device wait that nothing satisfies (FC_ERR_TIMEOUT expected)."""
    return int(load_library().fc_selftest_wait_timeout(ctx.ptr, int(wait_limit)))


FC_PROBE_L2_READ, FC_PROBE_SMEM_ATOMIC, FC_PROBE_AND_POPC = 0, 1, 2


def fc_probe_rate(kind: int, size: int = 0, stream=None) -> float:
    """Rate of one on-chip unit on the current device (fc_probe_rate in
    include/fc.h): bytes/s, atomics/s or words/s."""
    out = ctypes.c_double(0.0)
    _check(load_library().fc_probe_rate(int(kind), int(size), ctypes.byref(out), _stream_ptr(stream)))
    return float(out.value)


def fc_count_sorted_noalloc(D, arities, vars_, table, stream=None):
    """One table by sort + run-length with the library's fixed scratch (no
    allocation).  D: CUDA uint8 tensor (n, ld) column-major, rows of at least
    m instances; table: CUDA int32 tensor of prod(arities[vars]) cells.  The
    call is asynchronous on `stream`.  Arguments the C call cannot check
    (device buffer sizes, dtypes, devices, the length of `arities`) are
    checked here before anything is enqueued."""
    if not (_is_cuda(D) and _is_cuda(table)):
        raise FcError(FC_ERR_ARG, "fc_count_sorted_noalloc needs CUDA tensors for D and table")
    import torch
    if D.dtype != torch.uint8 or D.dim() != 2 or (D.shape[1] > 1 and D.stride(1) != 1):
        raise FcError(FC_ERR_ARG, "D must be a 2-D uint8 tensor whose instances are contiguous (stride(1) == 1)")
    if table.dtype != torch.int32 or not table.is_contiguous():
        raise FcError(FC_ERR_ARG, "table must be a contiguous int32 tensor")
    cur = torch.cuda.current_device()
    if D.device.index != cur or table.device.index != cur:
        raise FcError(FC_ERR_ARG, f"D and table must be on the current device (cuda:{cur})")
    ar, v = _host(arities, np.int32), _host(vars_, np.int32)
    n, m = int(D.shape[0]), int(D.shape[1])
    ld = int(D.stride(0)) if n > 1 else m
    if ar.ndim != 1 or len(ar) < n:
        raise FcError(FC_ERR_ARG, f"arities holds {ar.size} values for {n} variables")
    if v.ndim != 1 or np.any(v < 0) or np.any(v >= n):
        raise FcError(FC_ERR_ARG, "a variable id is outside 0..n-1")
    cells = 1
    for x in v:
        cells *= int(ar[x])
    if table.numel() < cells:
        raise FcError(FC_ERR_SIZE, f"table holds {table.numel()} cells, the query needs {cells}")
    _check(load_library().fc_count_sorted_noalloc(_ptr(D), n, m, ld, _ptr(ar, _i32p), _ptr(v, _i32p), len(v),
                                                  _ptr(table), _stream_ptr(stream)))


# ----------------------------------------------------------------- helpers

def fc_arities(ctx: Handle) -> np.ndarray:
    """Arities the context was loaded with (all 1 for transaction data)."""
    return ctx.arities
