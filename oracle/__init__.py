"""TEST INFRASTRUCTURE ONLY: ctypes wrapper around the C oracle (``oracle.c``).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library never loads it.

``run(workload)`` evaluates a :class:`datagen.workloads.Workload` and returns an
:class:`OracleResult` with the groups sorted ascending by packed key.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_I32, ORC_I64, ORC_U8 = 0, 1, 2
ORC_SUM, ORC_SUM_MUL_SUB, ORC_COUNT, ORC_AVG = 0, 1, 2, 3
STATUS = {0: "ok", 1: "invalid", 4: "dup_key", 8: "range", 9: "nomem"}
_TYPES = {np.dtype(np.int32): ORC_I32, np.dtype(np.int64): ORC_I64, np.dtype(np.uint8): ORC_U8}


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle status {code} ({STATUS.get(code, '?')})")
        self.code = code
        self.status = STATUS.get(code, "?")


class _Column(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("data", ctypes.c_void_p)]


class _Agg(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("col_a", ctypes.c_int32), ("col_b", ctypes.c_int32),
                ("k", ctypes.c_int64)]


class _Query(ctypes.Structure):
    _fields_ = [
        ("n_fact", ctypes.c_uint64), ("n_fact_cols", ctypes.c_int32),
        ("fact", ctypes.POINTER(_Column)),
        ("n_dim", ctypes.c_uint64), ("n_dim_cols", ctypes.c_int32),
        ("dim", ctypes.POINTER(_Column)),
        ("filter_col", ctypes.c_int32), ("filter_lo", ctypes.c_int64), ("filter_hi", ctypes.c_int64),
        ("join_fact_col", ctypes.c_int32), ("join_dim_col", ctypes.c_int32),
        ("n_group", ctypes.c_int32), ("group_side", ctypes.c_int32 * 4),
        ("group_col", ctypes.c_int32 * 4), ("group_bits", ctypes.c_int32 * 4),
        ("n_agg", ctypes.c_int32), ("aggs", _Agg * 8),
        ("dim_filter_col", ctypes.c_int32), ("dim_filter_lo", ctypes.c_int64), ("dim_filter_hi", ctypes.c_int64),
        ("n_extra_dims", ctypes.c_int32), ("n_xdim", ctypes.c_uint64 * 3), ("n_xdim_cols", ctypes.c_int32 * 3),
        ("xdim", ctypes.POINTER(_Column) * 3), ("xjoin_fact_col", ctypes.c_int32 * 3),
        ("xjoin_dim_col", ctypes.c_int32 * 3), ("xdim_filter_col", ctypes.c_int32 * 3),
        ("xdim_filter_lo", ctypes.c_int64 * 3), ("xdim_filter_hi", ctypes.c_int64 * 3),
        ("join_many", ctypes.c_int32),
    ]


class _Result(ctypes.Structure):
    _fields_ = [("n_groups", ctypes.c_uint64), ("keys", ctypes.POINTER(ctypes.c_uint64)),
                ("counts", ctypes.POINTER(ctypes.c_int64)), ("sums", ctypes.POINTER(ctypes.c_uint64)),
                ("avgs", ctypes.POINTER(ctypes.c_double))]


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.orc_run.restype = ctypes.c_int32
            lib.orc_run.argtypes = [ctypes.POINTER(_Query), ctypes.POINTER(_Result)]
            lib.orc_free.restype = None
            lib.orc_free.argtypes = [ctypes.POINTER(_Result)]
            lib.orc_i128_to_double.restype = ctypes.c_double
            lib.orc_i128_to_double.argtypes = [ctypes.c_uint64, ctypes.c_int64]
            _lib = lib
    return _lib


@dataclass
class OracleResult:
    keys: np.ndarray        # uint64 [G], ascending
    counts: np.ndarray      # int64 [G]
    sums: np.ndarray        # uint64 [G, A, 2]: int128 as (lo, hi) words
    avgs: np.ndarray        # float64 [G, A]
    aggs: list

    @property
    def n_groups(self) -> int:
        return int(self.keys.size)

    def sum_int(self, g: int, a: int) -> int:
        lo, hi = int(self.sums[g, a, 0]), int(self.sums[g, a, 1])
        v = (hi << 64) | lo
        return v - (1 << 128) if v >= 1 << 127 else v


def _columns(table: dict):
    names = list(table.keys())
    arrs = [np.ascontiguousarray(table[n]) for n in names]
    cols = (_Column * max(1, len(arrs)))()
    for i, a in enumerate(arrs):
        cols[i].type = _TYPES[a.dtype]
        cols[i].data = a.ctypes.data
    return names, arrs, cols


def run(wl) -> OracleResult:
    """Evaluate a workload's query over its tables; raises OracleError."""
    return run_query(wl.fact, wl.dim, wl.query, getattr(wl, "extra_dims", None))


def run_query(fact: dict, dim: dict | None, query: dict, extra_dims: list | None = None) -> OracleResult:
    """query: filter, join (with many=True: repeated build keys, fan-out), group,
    aggs, optional dim_filter; a star join adds
    extra_joins = [dict(fact_col, dim_col, optional dim_filter), ...] over the
    tables extra_dims, whose group fields use sides "dim1", "dim2", "dim3"."""
    lib = _load()
    fnames, farrs, fcols = _columns(fact)
    dnames, darrs, dcols = _columns(dim if dim is not None else {})
    xjoins = query.get("extra_joins") or []
    xd = [_columns(t) for t in (extra_dims or [])]
    n_fact = len(farrs[0]) if farrs else 0
    n_dim = len(darrs[0]) if darrs else 0
    q = _Query()
    q.n_fact, q.n_fact_cols, q.fact = n_fact, len(farrs), fcols
    q.n_dim, q.n_dim_cols, q.dim = n_dim, len(darrs), dcols
    f = query.get("filter")
    if f is None:
        q.filter_col, q.filter_lo, q.filter_hi = -1, 0, 0
    else:
        q.filter_col, q.filter_lo, q.filter_hi = fnames.index(f["col"]), f["lo"], f["hi"]
    j = query.get("join")
    if j is None:
        q.join_fact_col, q.join_dim_col = -1, -1
    else:
        q.join_fact_col, q.join_dim_col = fnames.index(j["fact_col"]), dnames.index(j["dim_col"])
        q.join_many = 1 if j.get("many") else 0
    df = query.get("dim_filter")
    if df is None:
        q.dim_filter_col, q.dim_filter_lo, q.dim_filter_hi = -1, 0, 0
    else:
        q.dim_filter_col, q.dim_filter_lo, q.dim_filter_hi = dnames.index(df["col"]), df["lo"], df["hi"]
    if len(xjoins) > len(xd):
        raise ValueError("extra_joins needs one table per join in extra_dims")
    q.n_extra_dims = len(xjoins)
    for j, xj in enumerate(xjoins):
        names, arrs, cols = xd[j]
        q.n_xdim[j] = len(arrs[0]) if arrs else 0
        q.n_xdim_cols[j] = len(arrs)
        q.xdim[j] = cols
        q.xjoin_fact_col[j] = fnames.index(xj["fact_col"])
        q.xjoin_dim_col[j] = names.index(xj["dim_col"])
        xf = xj.get("dim_filter")
        q.xdim_filter_col[j] = -1 if xf is None else names.index(xf["col"])
        q.xdim_filter_lo[j], q.xdim_filter_hi[j] = (0, 0) if xf is None else (xf["lo"], xf["hi"])
    sides = {"fact": (0, fnames), "dim": (1, dnames)}
    for j in range(len(xjoins)):
        sides[f"dim{j + 1}"] = (2 + j, xd[j][0])
    q.n_group = len(query["group"])
    for i, (side, col, bits) in enumerate(query["group"]):
        q.group_side[i], names = sides[side]
        q.group_col[i] = names.index(col)
        q.group_bits[i] = bits
    q.n_agg = len(query["aggs"])
    for i, ag in enumerate(query["aggs"]):
        kind = ag[0]
        if kind == "sum":
            q.aggs[i].kind, q.aggs[i].col_a = ORC_SUM, fnames.index(ag[1])
        elif kind == "avg":
            q.aggs[i].kind, q.aggs[i].col_a = ORC_AVG, fnames.index(ag[1])
        elif kind == "count":
            q.aggs[i].kind = ORC_COUNT
        elif kind == "sum_mul_sub":
            q.aggs[i].kind = ORC_SUM_MUL_SUB
            q.aggs[i].col_a, q.aggs[i].k, q.aggs[i].col_b = fnames.index(ag[1]), ag[2], fnames.index(ag[3])
        else:
            raise ValueError(kind)
    res = _Result()
    keep = (farrs, darrs, xd)   # the column arrays must outlive the call
    rc = lib.orc_run(ctypes.byref(q), ctypes.byref(res))
    del keep
    if rc != 0:
        raise OracleError(rc)
    try:
        g, a = int(res.n_groups), q.n_agg
        keys = np.ctypeslib.as_array(res.keys, shape=(max(g, 1),))[:g].copy()
        counts = np.ctypeslib.as_array(res.counts, shape=(max(g, 1),))[:g].copy()
        sums = np.ctypeslib.as_array(res.sums, shape=(max(g, 1) * max(a, 1) * 2,))
        sums = sums[: g * a * 2].copy().reshape(g, a, 2)
        avgs = np.ctypeslib.as_array(res.avgs, shape=(max(g, 1) * max(a, 1),))[: g * a].copy()
        avgs = avgs.reshape(g, a)
    finally:
        lib.orc_free(ctypes.byref(res))
    return OracleResult(keys, counts, sums, avgs, list(query["aggs"]))


def i128_to_double(v: int) -> float:
    """(double) of a 128-bit integer, by the C conversion the oracle uses."""
    v &= (1 << 128) - 1
    hi = v >> 64
    hi = hi - (1 << 64) if hi >= 1 << 63 else hi
    return _load().orc_i128_to_double(v & ((1 << 64) - 1), hi)
