"""Seeded, counter-based input generator (ctypes wrapper over ``gen.c``).

Input data only: this package holds no filter, join, grouping or aggregation
arithmetic.  The oracle and the CUDA path both take their inputs from here and
share nothing else.  See ``gen.c`` for the generator definitions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libdatagen.so")
_lock = threading.Lock()
_lib = None

# column kinds (gen.c)
UNIFORM, IOTA, PERM, PERM_DIV, RAW64, MODULAR = range(6)
_TYPES = {np.dtype(np.int32): 0, np.dtype(np.int64): 1, np.dtype(np.uint8): 2}


def build(force: bool = False) -> str:
    """Compile gen.c into libdatagen.so beside it (host C, OpenMP)."""
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            u64, i64, i32, dbl, vp = (ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_void_p)
            lib.dg_stream_key.restype = u64
            lib.dg_stream_key.argtypes = [u64, u64]
            lib.dg_fill.restype = i32
            lib.dg_fill.argtypes = [u64, u64, i32, i32, i64, i64, i64, i64, u64, u64, vp]
            lib.dg_fill_index.restype = i32
            lib.dg_fill_index.argtypes = [u64, u64, i32, u64, vp, u64, u64, vp]
            lib.dg_zipf_cdf.restype = i32
            lib.dg_zipf_cdf.argtypes = [dbl, u64, vp]
            lib.dg_gather.restype = i32
            lib.dg_gather.argtypes = [vp, i32, vp, u64, vp]
            lib.dg_lognormal.restype = i32
            lib.dg_lognormal.argtypes = [u64, u64, dbl, dbl, i64, i64, u64, vp]
            lib.dg_loguniform.restype = i32
            lib.dg_loguniform.argtypes = [u64, u64, i64, i64, u64, vp]
            lib.dg_raw_at.restype = i32
            lib.dg_raw_at.argtypes = [u64, u64, vp, u64, vp]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def fill(seed, stream, kind, dtype, n, a=0, b=0, c=0, mult=1, row0=0, out=None) -> np.ndarray:
    """Rows row0..row0+n-1 of one generated column (see gen.c for ``kind``)."""
    dtype = np.dtype(dtype)
    if out is None:
        out = np.empty(n, dtype=dtype)
    assert out.dtype == dtype and out.flags.c_contiguous and out.size >= n
    rc = _load().dg_fill(seed, stream, kind, _TYPES[dtype], a, b, c, mult, row0, n, _ptr(out))
    if rc != 0:
        raise ValueError(f"dg_fill rejected kind={kind} a={a} b={b}")
    return out


def uniform(seed, stream, dtype, n, lo, hi, mult=1, row0=0, out=None):
    return fill(seed, stream, UNIFORM, dtype, n, a=lo, b=hi, mult=mult, row0=row0, out=out)


def zipf_cdf(s: float, n: int) -> np.ndarray:
    cdf = np.empty(n, dtype=np.float64)
    if _load().dg_zipf_cdf(s, n, _ptr(cdf)) != 0:
        raise ValueError("bad zipf size")
    return cdf


def index(seed, stream, n_target, n, cdf=None, row0=0) -> np.ndarray:
    """Row indices into a table of ``n_target`` rows: uniform, or Zipf when a cdf is given."""
    out = np.empty(n, dtype=np.int64)
    dist = 0 if cdf is None else 1
    cp = 0 if cdf is None else _ptr(cdf)
    if _load().dg_fill_index(seed, stream, dist, n_target, cp, row0, n, _ptr(out)) != 0:
        raise ValueError("bad index arguments")
    return out


def gather(table: np.ndarray, idx: np.ndarray) -> np.ndarray:
    table = np.ascontiguousarray(table)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(idx.size, dtype=table.dtype)
    _load().dg_gather(_ptr(table), _TYPES[table.dtype], _ptr(idx), idx.size, _ptr(out))
    return out


def lognormal(seed, stream, mu, sigma, lo, hi, n) -> np.ndarray:
    out = np.empty(n, dtype=np.int64)
    _load().dg_lognormal(seed, stream, mu, sigma, lo, hi, n, _ptr(out))
    return out


def loguniform(seed, stream, lo, hi, n) -> np.ndarray:
    out = np.empty(n, dtype=np.int64)
    _load().dg_loguniform(seed, stream, lo, hi, n, _ptr(out))
    return out


def raw_at(seed, stream, idx: np.ndarray) -> np.ndarray:
    """RAW64 column values at arbitrary row indices."""
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(idx.size, dtype=np.int64)
    _load().dg_raw_at(seed, stream, _ptr(idx), idx.size, _ptr(out))
    return out
