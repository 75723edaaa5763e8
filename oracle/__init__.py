"""CPU oracle for counting queries and their scores (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_1804_04640_gb300`` never touches it and the two share no code.

The arithmetic lives in ``fc_oracle.c`` (plain loops, int64 counts, float64
scores, each function citing the passage of the paper it follows).  This file
compiles it with gcc into ``oracle/_build/liboracle.so`` on first use and
marshals numpy arrays through ctypes.  ctypes drops the GIL during a call, so
independent queries may be run from a thread pool.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fc_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain gcc, no vendor code)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    stale = (not os.path.exists(_OUT)) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_table.argtypes = [_u8p, ctypes.c_int64, ctypes.c_int32, _i32p, _i32p,
                                      ctypes.c_int32, _i64p]
            lib.orc_table.restype = ctypes.c_int
            lib.orc_count_assignment.argtypes = [_u8p, ctypes.c_int64, ctypes.c_int32, _i32p,
                                                 _i32p, ctypes.c_int32]
            lib.orc_count_assignment.restype = ctypes.c_int64
            for name in ("orc_ll",):
                getattr(lib, name).argtypes = [_i64p, ctypes.c_int64, ctypes.c_int32]
                getattr(lib, name).restype = ctypes.c_double
            lib.orc_mi.argtypes = [_i64p, ctypes.c_int64, ctypes.c_int32]
            lib.orc_mi.restype = ctypes.c_double
            lib.orc_mdl.argtypes = [_i64p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64]
            lib.orc_mdl.restype = ctypes.c_double
            lib.orc_bdeu.argtypes = [_i64p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double]
            lib.orc_bdeu.restype = ctypes.c_double
            lib.orc_support_rules.argtypes = [_u64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                              _i32p, ctypes.c_int32, _i64p, _i64p, _f64p]
            lib.orc_support_rules.restype = ctypes.c_int
            lib.orc_support_splits.argtypes = [_u64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                               _i32p, ctypes.c_int32, _i64p, _i64p, _f64p]
            lib.orc_support_splits.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


class OracleError(RuntimeError):
    pass


class DB:
    """The oracle's own row-major copy of a database ``D`` given as (n, m)."""

    def __init__(self, D: np.ndarray, arities):
        D = np.asarray(D, dtype=np.uint8)
        self.n, self.m = int(D.shape[0]), int(D.shape[1])
        self.rows = np.ascontiguousarray(D.T)
        self.arities = np.ascontiguousarray(np.asarray(arities, dtype=np.int32))

    def table(self, vars) -> np.ndarray:
        """Dense int64 table over ``vars`` (last variable fastest)."""
        lib = _load()
        v = np.ascontiguousarray(np.asarray(vars, dtype=np.int32))
        cells = int(np.prod([int(self.arities[x]) for x in v])) if len(v) else 1
        out = np.empty(cells, dtype=np.int64)
        rc = lib.orc_table(_p(self.rows, _u8p), self.m, self.n, _p(self.arities, _i32p),
                           _p(v, _i32p), len(v), _p(out, _i64p))
        if rc != 0:
            raise OracleError(f"orc_table failed with {rc}")
        return out

    def count_assignment(self, vars, states) -> int:
        lib = _load()
        v = np.ascontiguousarray(np.asarray(vars, dtype=np.int32))
        s = np.ascontiguousarray(np.asarray(states, dtype=np.int32))
        return int(lib.orc_count_assignment(_p(self.rows, _u8p), self.m, self.n,
                                            _p(v, _i32p), _p(s, _i32p), len(v)))

    def score(self, child: int, parents, kind: str, ess: float = 1.0) -> float:
        """Score of ``child`` given ``parents``: table over (parents..., child)."""
        t = self.table(list(parents) + [child])
        r = int(self.arities[child])
        return score_table(t, len(t) // r, r, kind, ess, self.m)


def score_table(table: np.ndarray, q: int, r: int, kind: str, ess: float = 1.0,
                m: int | None = None) -> float:
    lib = _load()
    t = np.ascontiguousarray(np.asarray(table, dtype=np.int64))
    if m is None:
        m = int(t.sum())
    if kind == "ll":
        return float(lib.orc_ll(_p(t, _i64p), q, r))
    if kind == "mdl":
        return float(lib.orc_mdl(_p(t, _i64p), q, r, m))
    if kind == "bdeu":
        return float(lib.orc_bdeu(_p(t, _i64p), q, r, ess))
    if kind == "mi":
        return float(lib.orc_mi(_p(t, _i64p), q, r))
    raise ValueError(kind)


def support_rules(bitmaps: np.ndarray, m: int, items):
    """(supp(S), [supp(S minus item t)], [conf((S minus item t) => item t)])."""
    lib = _load()
    b = np.ascontiguousarray(np.asarray(bitmaps, dtype=np.uint64))
    it = np.ascontiguousarray(np.asarray(items, dtype=np.int32))
    k = len(it)
    supp = np.zeros(1, dtype=np.int64)
    sub = np.zeros(max(k, 1), dtype=np.int64)
    conf = np.zeros(max(k, 1), dtype=np.float64)
    rc = lib.orc_support_rules(_p(b, _u64p), b.shape[1], m, b.shape[0], _p(it, _i32p), k,
                               _p(supp, _i64p), _p(sub, _i64p), _p(conf, _f64p))
    if rc != 0:
        raise OracleError(f"orc_support_rules failed with {rc}")
    return int(supp[0]), sub[:k].copy(), conf[:k].copy()


def support_splits(bitmaps: np.ndarray, m: int, items):
    """(supp(S), [supp(A)], [conf(A => S minus A)]) for every antecedent mask
    A = 1 .. 2^k - 2 over the positions of ``items``."""
    lib = _load()
    b = np.ascontiguousarray(np.asarray(bitmaps, dtype=np.uint64))
    it = np.ascontiguousarray(np.asarray(items, dtype=np.int32))
    k = len(it)
    n = max((1 << k) - 2, 1)
    supp = np.zeros(1, dtype=np.int64)
    sub = np.zeros(n, dtype=np.int64)
    conf = np.zeros(n, dtype=np.float64)
    rc = lib.orc_support_splits(_p(b, _u64p), b.shape[1], m, b.shape[0], _p(it, _i32p), k,
                                _p(supp, _i64p), _p(sub, _i64p), _p(conf, _f64p))
    if rc != 0:
        raise OracleError(f"orc_support_splits failed with {rc}")
    nn = max((1 << k) - 2, 0)
    return int(supp[0]), sub[:nn].copy(), conf[:nn].copy()
