"""Python access to the C oracle (oracle.c): TEST INFRASTRUCTURE ONLY.

Plain, slow, row-at-a-time statements of what the Crystal GPU operators compute.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm
import this package.  It never imports the GPU package and the GPU package never
imports it; the only code both sides use is the seeded input generator ``datagen``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

MAX_COLS, MAX_PREDS, MAX_JOINS, MAX_DIM_PREDS = 16, 8, 4, 4
AGG_OPS = {"sum": 0, "mul": 1, "sub": 2, "add": 3}


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C, no SIMD intrinsics, no FMA contraction)."""
    stale = force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                           os.path.getmtime(os.path.join(_HERE, "oracle.h"))))
    if stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                               "-std=c11", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _DimPred(C.Structure):
    _fields_ = [("col", C.c_void_p), ("lo", C.c_int32), ("hi", C.c_int32)]


class _Join(C.Structure):
    _fields_ = [("fk_col", C.c_int32), ("dim_keys", C.c_void_p), ("dim_rows", C.c_int64),
                ("n_preds", C.c_int32), ("preds", _DimPred * MAX_DIM_PREDS),
                ("group_attr", C.c_void_p), ("group_card", C.c_int32)]


class _FactPred(C.Structure):
    _fields_ = [("col", C.c_int32), ("lo", C.c_int32), ("hi", C.c_int32)]


class _Plan(C.Structure):
    _fields_ = [("cols", C.c_void_p * MAX_COLS), ("n_cols", C.c_int32), ("n_rows", C.c_int64),
                ("n_preds", C.c_int32), ("preds", _FactPred * MAX_PREDS),
                ("n_joins", C.c_int32), ("joins", _Join * MAX_JOINS),
                ("agg_op", C.c_int32), ("agg_a", C.c_int32), ("agg_b", C.c_int32)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        p, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        L.orc_select.argtypes = [p, i64, i32, i32, p]
        L.orc_select.restype = i64
        L.orc_select_mt.argtypes = [p, i64, i32, i32, p, C.c_int]
        L.orc_select_mt.restype = i64
        L.orc_tile_scan.argtypes = [p, i32, i32, p, p, p, p]
        L.orc_project.argtypes = [p, p, i64, C.c_float, C.c_float, C.c_int, p]
        L.orc_project_mt.argtypes = [p, p, i64, C.c_float, C.c_float, C.c_int, p, C.c_int]
        L.orc_join_sum.argtypes = [p, p, i64, p, p, i64, p]
        L.orc_join_sum.restype = i64
        L.orc_join_sum_mt.argtypes = [p, p, i64, p, p, i64, p, C.c_int]
        L.orc_join_sum_mt.restype = i64
        L.orc_sort.argtypes = [p, p, i64, p, p]
        L.orc_run_plan.argtypes = [C.POINTER(_Plan), p, p]
        L.orc_run_plan.restype = C.c_int
        L.orc_run_plan_mt.argtypes = [C.POINTER(_Plan), p, p, C.c_int]
        L.orc_run_plan_mt.restype = C.c_int
        L.orc_hardware_threads.restype = C.c_int
        _lib = L
    return _lib


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def hardware_threads() -> int:
    return int(lib().orc_hardware_threads())


def select(x, lo: int, hi: int, threads: int = 1) -> np.ndarray:
    """Rows of x with lo <= x <= hi, in input order."""
    x = _i32(x)
    out = np.empty(max(1, x.size), dtype=np.int32)
    if threads > 1:
        n = lib().orc_select_mt(_ptr(x), x.size, lo, hi, _ptr(out), threads)
    else:
        n = lib().orc_select(_ptr(x), x.size, lo, hi, _ptr(out))
    return out[:n].copy()


def tile_scan(flags, threads: int, items: int):
    f = np.ascontiguousarray(flags, dtype=np.uint8)
    assert f.size == threads * items
    counts = np.empty(threads, np.int32)
    offsets = np.empty(threads, np.int32)
    total = np.zeros(1, np.int32)
    order = np.full(threads * items, -1, np.int32)
    lib().orc_tile_scan(_ptr(f), threads, items, _ptr(counts), _ptr(offsets), _ptr(total),
                        _ptr(order))
    return counts, offsets, int(total[0]), order[: int(total[0])]


def project(x1, x2, a: float, b: float, op: int = 0, threads: int = 1) -> np.ndarray:
    x1, x2 = _f32(x1), _f32(x2)
    assert x1.shape == x2.shape
    y = np.empty_like(x1)
    if threads > 1:
        lib().orc_project_mt(_ptr(x1), _ptr(x2), x1.size, a, b, op, _ptr(y), threads)
    else:
        lib().orc_project(_ptr(x1), _ptr(x2), x1.size, a, b, op, _ptr(y))
    return y


def join_sum(bkeys, bvals, fk, payload, threads: int = 1):
    """(SUM(payload * value) over matching pairs, number of matching probe rows)."""
    bk, bv, f, pl = _i32(bkeys), _i32(bvals), _i32(fk), _i32(payload)
    assert bk.size == bv.size and f.size == pl.size
    m = np.zeros(1, np.int64)
    s = lib().orc_join_sum_mt(_ptr(bk), _ptr(bv), bk.size, _ptr(f), _ptr(pl), f.size, _ptr(m),
                              max(1, threads))
    if m[0] < 0:
        raise ValueError("duplicate build key")
    return int(s), int(m[0])


def sort(keys, vals):
    k, v = _i32(keys), _i32(vals)
    ko, vo = np.empty_like(k), np.empty_like(v)
    lib().orc_sort(_ptr(k), _ptr(v), k.size, _ptr(ko), _ptr(vo))
    return ko, vo


def run_plan_raw(fact_cols: list, preds: list, joins: list, agg: tuple, threads: int = 1):
    """General select-join-group-by.

    fact_cols: list of int32 arrays (same length).  preds: [(col_idx, lo, hi)].
    joins: [{"fk_col": idx, "keys": arr, "preds": [(arr, lo, hi)], "group": arr|None,
    "card": int}].  agg: (op_name, a_idx, b_idx|None).  Returns (sums, counts).
    """
    keep = []
    plan = _Plan()
    cols = [_i32(c) for c in fact_cols]
    keep += cols
    n_rows = cols[0].size if cols else 0
    assert all(c.size == n_rows for c in cols)
    for i, c in enumerate(cols):
        plan.cols[i] = c.ctypes.data
    plan.n_cols, plan.n_rows = len(cols), n_rows
    plan.n_preds = len(preds)
    for k, (ci, lo, hi) in enumerate(preds):
        plan.preds[k] = _FactPred(ci, lo, hi)
    plan.n_joins = len(joins)
    groups = 1
    for j, jn in enumerate(joins):
        keys = _i32(jn["keys"])
        keep.append(keys)
        js = plan.joins[j]
        js.fk_col = jn["fk_col"]
        js.dim_keys = keys.ctypes.data
        js.dim_rows = keys.size
        js.n_preds = len(jn.get("preds", []))
        for k, (arr, lo, hi) in enumerate(jn.get("preds", [])):
            arr = _i32(arr)
            keep.append(arr)
            js.preds[k] = _DimPred(arr.ctypes.data, lo, hi)
        if jn.get("group") is not None:
            g = _i32(jn["group"])
            keep.append(g)
            js.group_attr = g.ctypes.data
            js.group_card = int(jn["card"])
            groups *= int(jn["card"])
        else:
            js.group_attr = None
            js.group_card = 1
    op, a, b = agg
    plan.agg_op, plan.agg_a, plan.agg_b = AGG_OPS[op], a, (b if b is not None else 0)
    sums = np.zeros(groups, np.int64)
    counts = np.zeros(groups, np.int64)
    rc = lib().orc_run_plan_mt(C.byref(plan), _ptr(sums), _ptr(counts), max(1, threads))
    if rc != 0:
        raise ValueError("invalid plan")
    return sums, counts


def q1_run(fact: dict, dim: dict, year: int = 3, threads: int = 1) -> int:
    """Fused filter-probe-aggregate query: yr == year AND a < 25 AND 1 <= b <= 3,
    SUM(c * b) over fact rows whose fk names a dimension row."""
    cols = [fact["fk"], fact["a"], fact["b"], fact["c"]]
    joins = [{"fk_col": 0, "keys": dim["key"], "preds": [(dim["yr"], year, year)],
              "group": None, "card": 1}]
    sums, _ = run_plan_raw(cols, [(1, -(1 << 31), 24), (2, 1, 3)], joins, ("mul", 3, 2),
                           threads)
    return int(sums[0])


def ss_run(tables: dict, query: dict, threads: int = 1, fact_rows: int | None = None):
    """A served star-schema query (datagen.ss_query format) -> (sums, counts)."""
    import datagen
    fact, dims = tables["fact"], tables["dims"]
    names = list(datagen.SS_FACT_COLS)
    n = fact[names[0]].size if fact_rows is None else fact_rows
    cols = [fact[c][:n] for c in names]
    preds = [(names.index(c), lo, hi) for (c, lo, hi) in query["fact_preds"]]
    joins = []
    for jn in query["joins"]:
        d = dims[jn["dim"]]
        spec = datagen.SS_DIMS[jn["dim"]]
        joins.append({
            "fk_col": names.index(spec["fk"]), "keys": d["key"],
            "preds": [(d[a], lo, hi) for (a, lo, hi) in jn["filters"]],
            "group": d[jn["group"]] if jn["group"] is not None else None,
            "card": spec["attrs"][jn["group"]] if jn["group"] is not None else 1,
        })
    op, a, b = query["agg"]
    agg = (op, names.index(a), names.index(b) if b is not None else None)
    return run_plan_raw(cols, preds, joins, agg, threads)
