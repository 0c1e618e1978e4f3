"""Exact relational oracle (plain C in ``oracle.c``) with a numpy interface.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Semantics (plain SQL, Sec. 2 "Query Processor", Sec. 4, Sec. 5.2):
  filter(cols, preds)          -> int32 row ids, ascending
  groupby(keys, aggs, sel)     -> (key columns, aggregate columns), groups in
                                  ascending key order
  join(bkey, pkey, bsel, psel) -> (probe row ids, build row ids) in probe order
  topk(vals, keys, k)          -> value desc, key asc
  sort_pairs(keys, vals)       -> stable by unsigned key

filter / groupby / join take parallel=True to run the OpenMP row-partitioned
versions in oracle.c (same results; used to time the CPU baseline on all host
cores, threads() of them).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None

DT = {np.dtype(np.int8): 0, np.dtype(np.int32): 1, np.dtype(np.int64): 2, np.dtype(np.uint8): 3}
CMP = {"<": 0, "<=": 1, ">": 2, ">=": 3, "==": 4, "!=": 5}
AGG = {"count": 0, "sum": 1, "sum_mul_kminus": 2, "avg": 3, "min": 4, "max": 5}

_p = C.c_void_p
_i64 = C.c_int64


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.orc_filter.restype = _i64
        L.orc_filter.argtypes = [_i64, C.c_int, _p, _p, _p, _p, _p]
        L.orc_groupby.restype = _i64
        L.orc_groupby.argtypes = [_i64, _p, _i64, C.c_int, _p, _p, C.c_int, _p, _p, _p, _p, _p, _p, _p, _p, _i64]
        L.orc_join.restype = _i64
        L.orc_join.argtypes = [_i64, _p, _p, _i64, _i64, _p, _p, _i64, _p, _p, _i64, _p]
        L.orc_topk.restype = _i64
        L.orc_topk.argtypes = [_i64, _p, _p, _i64, _p, _p]
        L.orc_sort_pairs.restype = None
        L.orc_sort_pairs.argtypes = [_i64, _p, _p, _p, _p]
        L.orc_avg_round.restype = _i64
        L.orc_avg_round.argtypes = [_i64, _i64]
        L.orc_filter_omp.restype = _i64
        L.orc_filter_omp.argtypes = L.orc_filter.argtypes
        L.orc_groupby_omp.restype = _i64
        L.orc_groupby_omp.argtypes = L.orc_groupby.argtypes
        L.orc_join_omp.restype = _i64
        L.orc_join_omp.argtypes = L.orc_join.argtypes
        L.orc_omp_threads.restype = C.c_int
        L.orc_omp_threads.argtypes = []
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _ptr_array(arrs):
    return (C.c_void_p * max(1, len(arrs)))(*[a.ctypes.data for a in arrs])


def _int_array(vals, ctype=C.c_int):
    return (ctype * max(1, len(vals)))(*vals)


def threads() -> int:
    """Threads the parallel oracle functions use (OpenMP's maximum)."""
    return int(lib().orc_omp_threads())


def filter(preds, n: int, parallel: bool = False) -> np.ndarray:
    """preds: list of (column array, op string, integer literal)."""
    cols = [np.ascontiguousarray(c) for c, _, _ in preds]
    out = np.empty(max(1, n), dtype=np.int32)
    fn = lib().orc_filter_omp if parallel else lib().orc_filter
    m = fn(n, len(preds), _ptr_array(cols), _int_array([DT[c.dtype] for c in cols]),
                         _int_array([CMP[o] for _, o, _ in preds]),
                         _int_array([int(v) for _, _, v in preds], C.c_int64), _ptr(out))
    return out[:m].copy()


def avg_round(s: int, c: int) -> int:
    return int(lib().orc_avg_round(int(s), int(c)))


def groupby(keys, aggs, n: int, sel=None, parallel: bool = False):
    """keys: list of key column arrays.
    aggs: list of tuples (op, a, b, k) with op in AGG; a/b arrays or None.
    Returns (key matrix int64 [G, nkeys], agg matrix int64 [G, naggs])."""
    keys = [np.ascontiguousarray(k) for k in keys]
    dummy = np.zeros(1, np.int64)
    acols = [np.ascontiguousarray(a[1]) if a[1] is not None else dummy for a in aggs]
    bcols = [np.ascontiguousarray(a[2]) if a[2] is not None else dummy for a in aggs]
    ks = [int(a[3]) if a[3] is not None else 0 for a in aggs]
    selc = np.ascontiguousarray(sel, dtype=np.int32) if sel is not None else None
    m = len(selc) if selc is not None else n
    cap = max(1, m)
    ok = np.empty((cap, max(1, len(keys))), np.int64)
    oa = np.empty((cap, max(1, len(aggs))), np.int64)
    fn = lib().orc_groupby_omp if parallel else lib().orc_groupby
    g = fn(n, _ptr(selc), m, len(keys), _ptr_array(keys), _int_array([DT[k.dtype] for k in keys]),
                          len(aggs), _int_array([AGG[a[0]] for a in aggs]), _ptr_array(acols),
                          _int_array([DT[a.dtype] for a in acols]), _ptr_array(bcols),
                          _int_array([DT[b.dtype] for b in bcols]), _int_array(ks, C.c_int64),
                          _ptr(ok), _ptr(oa), cap)
    return ok[:g, : len(keys)].copy(), oa[:g, : len(aggs)].copy()


def join(bkey, pkey, bsel=None, psel=None, cap=None, parallel: bool = False):
    """Returns (probe row ids, build row ids, duplicate-build-key flag)."""
    bkey = np.ascontiguousarray(bkey, dtype=np.int32)
    pkey = np.ascontiguousarray(pkey, dtype=np.int32)
    bs = np.ascontiguousarray(bsel, dtype=np.int32) if bsel is not None else None
    ps = np.ascontiguousarray(psel, dtype=np.int32) if psel is not None else None
    L = lib()
    fn = L.orc_join_omp if parallel else L.orc_join
    dup = C.c_int(0)
    if cap is None:
        # count first, then fill
        cnt = fn(len(bkey), _ptr(bkey), _ptr(bs), len(bs) if bs is not None else 0,
                         len(pkey), _ptr(pkey), _ptr(ps), len(ps) if ps is not None else 0,
                         None, None, 0, C.byref(dup))
        cap = cnt
    op = np.empty(max(1, cap), np.int32)
    ob = np.empty(max(1, cap), np.int32)
    cnt = fn(len(bkey), _ptr(bkey), _ptr(bs), len(bs) if bs is not None else 0,
                     len(pkey), _ptr(pkey), _ptr(ps), len(ps) if ps is not None else 0,
                     _ptr(op), _ptr(ob), cap, C.byref(dup))
    m = min(cnt, cap)
    return op[:m].copy(), ob[:m].copy(), bool(dup.value)


def topk(vals, keys, k: int):
    vals = np.ascontiguousarray(vals, dtype=np.int64)
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    ov = np.empty(max(1, k), np.int64)
    okk = np.empty(max(1, k), np.int64)
    m = lib().orc_topk(len(vals), _ptr(vals), _ptr(keys), k, _ptr(ov), _ptr(okk))
    return ov[:m].copy(), okk[:m].copy()


def sort_pairs(keys, vals):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    vals = np.ascontiguousarray(vals, dtype=np.uint32)
    ok = np.empty_like(keys)
    ov = np.empty_like(vals)
    lib().orc_sort_pairs(len(keys), _ptr(keys), _ptr(vals), _ptr(ok), _ptr(ov))
    return ok, ov
