"""ctypes binding of ``libtheseus_gb.so`` (the C ABI in ``include/theseus_gb.h``).

Argument marshalling only: every step of a query runs in the library's CUDA
kernels.  The module-level ``tp_*`` names are the C functions themselves; the
small ``Engine`` / ``Table`` / ``Plan`` / ``Result`` classes wrap them with
numpy and torch conversions.  Loading fails loudly when the library has not
been built -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtheseus_gb.so")
_lock = threading.Lock()
_lib = None

# ----------------------------------------------------------------- constants
TP_OK, TP_E_INVALID, TP_E_POOL_EMPTY, TP_E_BUDGET, TP_E_DUP_KEY = 0, 1, 2, 3, 4
TP_E_TIMEOUT, TP_E_CUDA, TP_E_INTERNAL, TP_E_RANGE, TP_E_NOMEM = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "ok", 1: "invalid", 2: "pool_empty", 3: "budget", 4: "dup_key", 5: "timeout",
                6: "cuda", 7: "internal", 8: "range", 9: "nomem"}
TP_AGG_AUTO, TP_AGG_SHARED, TP_AGG_GLOBAL = 0, 1, 2
TP_I32, TP_I64, TP_U8 = 0, 1, 2
TP_HOST_PAGES, TP_DEVICE = 1, 2
TP_FLAG_TIME_KERNELS, TP_FLAG_NO_STAGED, TP_FLAG_EXACT_ONLY, TP_FLAG_NO_DIRECT_JOIN, TP_FLAG_NO_JIT = 1, 2, 4, 8, 16
TP_FLAG_NO_DIRECT_AGG, TP_FLAG_RAW_PAGES = 32, 64
TP_SIDE_FACT, TP_SIDE_DIM = 0, 1
TP_LIP_AUTO, TP_LIP_OFF, TP_LIP_ON = 0, 1, 2
TP_AGG_SUM, TP_AGG_SUM_MUL_SUB, TP_AGG_COUNT, TP_AGG_AVG = 0, 1, 2, 3
TP_SERVE_CACHE_DIM, TP_SERVE_BATCH = 1, 2
TP_COPY_PINNED_PER_BATCH = 1

_NP_TYPE = {np.dtype(np.int32): TP_I32, np.dtype(np.int64): TP_I64, np.dtype(np.uint8): TP_U8}
_TYPE_NP = {v: k for k, v in _NP_TYPE.items()}


class TPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS_NAMES.get(code, str(code))


# ----------------------------------------------------------------- structs
class tp_config(ctypes.Structure):
    _fields_ = [("page_bytes", ctypes.c_uint64), ("n_pages", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("device_budget_bytes", ctypes.c_uint64), ("prefetch_depth", ctypes.c_int32),
                ("cuda_device", ctypes.c_int32), ("batch_rows", ctypes.c_uint64),
                ("load_factor", ctypes.c_float), ("agg_strategy", ctypes.c_int32),
                ("compute_stream", ctypes.c_void_p)]


class tp_column_desc(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("type", ctypes.c_int32), ("scale", ctypes.c_int32)]


class tp_table_desc(ctypes.Structure):
    _fields_ = [("n_cols", ctypes.c_int32), ("cols", ctypes.POINTER(tp_column_desc)),
                ("batch_rows", ctypes.c_uint64)]


class tp_filter(ctypes.Structure):
    _fields_ = [("col", ctypes.c_int32), ("lo", ctypes.c_int64), ("hi", ctypes.c_int64)]


class tp_join(ctypes.Structure):
    _fields_ = [("fact_col", ctypes.c_int32), ("dim_col", ctypes.c_int32)]


class tp_group_field(ctypes.Structure):
    _fields_ = [("side", ctypes.c_int32), ("col", ctypes.c_int32), ("bits", ctypes.c_int32)]


class tp_agg(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("col_a", ctypes.c_int32), ("col_b", ctypes.c_int32),
                ("k", ctypes.c_int64)]


class tp_plan_desc(ctypes.Structure):
    _fields_ = [("fact", ctypes.c_void_p), ("dim", ctypes.c_void_p), ("filter", tp_filter),
                ("join", tp_join), ("n_group", ctypes.c_int32), ("group", tp_group_field * 4),
                ("n_agg", ctypes.c_int32), ("aggs", tp_agg * 8), ("agg_strategy", ctypes.c_int32),
                ("load_factor", ctypes.c_float), ("expected_groups", ctypes.c_uint64),
                ("join_partitions", ctypes.c_int32), ("dim_filter", tp_filter), ("dim_filter_on", ctypes.c_int32),
                ("lip", ctypes.c_int32), ("n_extra_dims", ctypes.c_int32), ("extra_dim", ctypes.c_void_p * 3),
                ("extra_join", tp_join * 3), ("extra_dim_filter", tp_filter * 3),
                ("extra_dim_filter_on", ctypes.c_int32 * 3), ("join_many", ctypes.c_int32)]


class tp_i128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_int64)]


class tp_stats(ctypes.Structure):
    _fields_ = [("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("peak_reserved", ctypes.c_uint64),
                ("retries", ctypes.c_uint64), ("pages_in_use", ctypes.c_uint32),
                ("pages_total", ctypes.c_uint32), ("agg_kernel_ms", ctypes.c_double),
                ("agg_kernel_launches", ctypes.c_uint64), ("agg_kernel_rows", ctypes.c_uint64),
                ("jit_compiles", ctypes.c_uint64), ("jit_failures", ctypes.c_uint64),
                ("jit_launches", ctypes.c_uint64), ("jit_compile_ms", ctypes.c_double),
                ("agg_split_passes", ctypes.c_uint64), ("lip_filters", ctypes.c_uint64),
                ("part_build_ms", ctypes.c_double), ("part_stream_ms", ctypes.c_double),
                ("part_spilled_ms", ctypes.c_double)]


class tp_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("budget_waits", ctypes.c_uint64), ("cache_hits", ctypes.c_uint64), ("cache_misses", ctypes.c_uint64),
                ("cache_evictions", ctypes.c_uint64), ("inflight_peak", ctypes.c_uint32), ("batches", ctypes.c_uint32)]


_vp, _u64, _i64, _i32, _u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
_PP = ctypes.POINTER(ctypes.c_void_p)

# name: (restype, argtypes) -- mirrors include/theseus_gb.h
SIGNATURES = {
    "tp_config_default": (None, [ctypes.POINTER(tp_config)]),
    "tp_init": (_i32, [ctypes.POINTER(tp_config), _PP]),
    "tp_shutdown": (None, [_vp]),
    "tp_page_alloc": (_i32, [_vp, ctypes.POINTER(_u32)]),
    "tp_page_free": (_i32, [_vp, _u32]),
    "tp_page_ptr": (_vp, [_vp, _u32]),
    "tp_page_bytes": (_u64, [_vp]),
    "tp_pages_free": (_u32, [_vp]),
    "tp_set_device_budget": (_i32, [_vp, _u64]),
    "tp_budget_query": (_i32, [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "tp_set_copy_options": (_i32, [_vp, _i32, _u32]),
    "tp_table_create": (_i32, [_vp, ctypes.POINTER(tp_table_desc), _PP]),
    "tp_table_append": (_i32, [_vp, _PP, _u64]),
    "tp_table_place": (_i32, [_vp, _i32]),
    "tp_table_wrap_device": (_i32, [_vp, ctypes.POINTER(tp_table_desc), _PP, _u64, _PP]),
    "tp_table_rows": (_u64, [_vp]),
    "tp_table_batches": (_u64, [_vp]),
    "tp_table_destroy": (None, [_vp]),
    "tp_plan_create": (_i32, [_vp, ctypes.POINTER(tp_plan_desc), _PP]),
    "tp_plan_destroy": (None, [_vp]),
    "tp_execute": (_i32, [_vp, _PP]),
    "tp_result_groups": (_u64, [_vp]),
    "tp_result_keys": (ctypes.POINTER(_u64), [_vp]),
    "tp_result_count": (ctypes.POINTER(_i64), [_vp]),
    "tp_result_sum": (ctypes.POINTER(tp_i128), [_vp, _i32]),
    "tp_result_avg": (ctypes.POINTER(ctypes.c_double), [_vp, _i32]),
    "tp_result_device_keys": (_vp, [_vp]),
    "tp_result_device_count": (_vp, [_vp]),
    "tp_result_device_sum": (_vp, [_vp, _i32]),
    "tp_result_device_avg": (_vp, [_vp, _i32]),
    "tp_result_free": (None, [_vp]),
    "tp_last_error": (ctypes.c_char_p, []),
    "tp_stats_get": (_i32, [_vp, ctypes.POINTER(tp_stats)]),
    "tp_debug_fail_next_alloc": (_i32, [_vp, _i32]),
    "tp_debug_pack_bits": (_i32, [_vp, _u64, _i32, _vp]),
    "tp_batch_create": (_i32, [_vp, _PP, _i32, ctypes.c_char_p, _PP]),
    "tp_batch_execute": (_i32, [_vp, _PP]),
    "tp_batch_last_ms": (ctypes.c_double, [_vp]),
    "tp_debug_batch_stall": (_i32, [_vp, _i32, _u64]),
    "tp_batch_destroy": (None, [_vp]),
    "tp_autotune": (_i32, [_vp, _PP, _i32, ctypes.c_char_p]),
    "tp_server_start": (_i32, [_vp, _i32, _i32, _u32, _PP]),
    "tp_submit": (_i32, [_vp, _vp, ctypes.POINTER(_u64)]),
    "tp_wait": (_i32, [_vp, _u64, _i64, _PP, ctypes.POINTER(_i64)]),
    "tp_server_stats_get": (_i32, [_vp, ctypes.POINTER(tp_server_stats)]),
    "tp_server_stop": (None, [_vp]),
    "tp_execute_noalloc": (_i32, [ctypes.POINTER(tp_plan_desc), _PP, ctypes.POINTER(_i32), _i32, _u64, _PP,
                                  ctypes.POINTER(_i32), _i32, _u64, _vp, _vp, _PP, _PP, ctypes.POINTER(_u64),
                                  _vp]),
}


def load():
    """Loads the CUDA library; raises if it is missing (build it first)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run paper_2508_05029_gb300.build.build() "
                                   "(the CUDA library is required; there is no CPU fallback)")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
                globals()[name] = fn
            _lib = lib
    return _lib


def _check(code: int):
    if code != TP_OK:
        raise TPError(code, (_lib.tp_last_error() or b"").decode(errors="replace"))


def last_error() -> str:
    return (load().tp_last_error() or b"").decode(errors="replace")


# ------------------------------------------------------------------ wrappers
class Engine:
    def __init__(self, page_bytes=64 << 20, n_pages=0, device_budget_bytes=0, prefetch_depth=2,
                 batch_rows=4 << 20, cuda_device=0, load_factor=0.5, agg_strategy=TP_AGG_AUTO,
                 compute_stream=None, flags=0):
        lib = load()
        cfg = tp_config()
        lib.tp_config_default(ctypes.byref(cfg))
        cfg.page_bytes, cfg.n_pages, cfg.device_budget_bytes = page_bytes, n_pages, device_budget_bytes
        cfg.prefetch_depth, cfg.batch_rows, cfg.cuda_device = prefetch_depth, batch_rows, cuda_device
        cfg.load_factor, cfg.agg_strategy = load_factor, agg_strategy
        cfg.compute_stream = compute_stream
        cfg.flags = flags
        h = ctypes.c_void_p()
        _check(lib.tp_init(ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h
        self.lib = lib

    def close(self):
        if self.h:
            self.lib.tp_shutdown(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def stats(self) -> dict:
        s = tp_stats()
        _check(self.lib.tp_stats_get(self.h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in tp_stats._fields_}

    def budget(self):
        r, c = _u64(), _u64()
        _check(self.lib.tp_budget_query(self.h, ctypes.byref(r), ctypes.byref(c)))
        return r.value, c.value

    def set_budget(self, nbytes: int):
        _check(self.lib.tp_set_device_budget(self.h, nbytes))

    def set_copy_options(self, prefetch_depth: int, pinned_per_batch: bool = False):
        _check(self.lib.tp_set_copy_options(self.h, prefetch_depth,
                                            TP_COPY_PINNED_PER_BATCH if pinned_per_batch else 0))

    def page_alloc(self) -> int:
        p = _u32()
        _check(self.lib.tp_page_alloc(self.h, ctypes.byref(p)))
        return p.value

    def page_free(self, p: int):
        _check(self.lib.tp_page_free(self.h, p))

    def pages_free(self) -> int:
        return self.lib.tp_pages_free(self.h)

    def fail_next_alloc(self, n: int):
        _check(self.lib.tp_debug_fail_next_alloc(self.h, n))

    # tables ---------------------------------------------------------------
    def _desc(self, names, dtypes, batch_rows=0):
        cols = (tp_column_desc * len(names))()
        keep = []
        for i, (n, dt) in enumerate(zip(names, dtypes)):
            b = n.encode()
            keep.append(b)
            cols[i].name, cols[i].type, cols[i].scale = b, _NP_TYPE[np.dtype(dt)], 0
        d = tp_table_desc(len(names), cols, batch_rows)
        return d, (cols, keep)

    def table_from_numpy(self, columns: dict, placement=TP_HOST_PAGES, batch_rows=0) -> "Table":
        names = list(columns)
        arrs = [np.ascontiguousarray(columns[n]) for n in names]
        d, keep = self._desc(names, [a.dtype for a in arrs], batch_rows)
        h = ctypes.c_void_p()
        _check(self.lib.tp_table_create(self.h, ctypes.byref(d), ctypes.byref(h)))
        t = Table(self, h, names)
        ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
        n = len(arrs[0]) if arrs else 0
        try:
            _check(self.lib.tp_table_append(h, ptrs, n))
            if placement == TP_DEVICE:
                _check(self.lib.tp_table_place(h, TP_DEVICE))
        except Exception:
            t.destroy()
            raise
        return t

    def table_from_chunks(self, chunks, batch_rows=0) -> "Table":
        """A host-page table appended chunk by chunk (dicts of equal-length
        numpy columns, the same names and dtypes in every chunk)."""
        t = None
        try:
            for columns in chunks:
                arrs = [np.ascontiguousarray(columns[n]) for n in columns]
                if t is None:
                    d, keep = self._desc(list(columns), [a.dtype for a in arrs], batch_rows)
                    h = ctypes.c_void_p()
                    _check(self.lib.tp_table_create(self.h, ctypes.byref(d), ctypes.byref(h)))
                    t = Table(self, h, list(columns))
                ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
                _check(self.lib.tp_table_append(t.h, ptrs, len(arrs[0])))
        except Exception:
            if t is not None:
                t.destroy()
            raise
        return t

    def table_from_torch(self, columns: dict) -> "Table":
        """Registers CUDA tensors without copying (they must outlive the table)."""
        import torch
        names = list(columns)
        ts = [columns[n] for n in names]
        for x in ts:
            assert x.is_cuda and x.is_contiguous() and x.dim() == 1
        tmap = {torch.int32: np.int32, torch.int64: np.int64, torch.uint8: np.uint8}
        d, keep = self._desc(names, [tmap[x.dtype] for x in ts])
        ptrs = (ctypes.c_void_p * len(ts))(*[x.data_ptr() for x in ts])
        h = ctypes.c_void_p()
        n = ts[0].numel() if ts else 0
        _check(self.lib.tp_table_wrap_device(self.h, ctypes.byref(d), ptrs, n, ctypes.byref(h)))
        t = Table(self, h, names)
        t._tensors = ts
        return t

    def table_from_pointers(self, columns: dict, nrows: int) -> "Table":
        """Registers device-accessible memory without copying: columns maps a
        name to (address, numpy dtype); the memory must outlive the table."""
        names = list(columns)
        d, keep = self._desc(names, [np.dtype(columns[n][1]) for n in names])
        ptrs = (ctypes.c_void_p * len(names))(*[int(columns[n][0]) for n in names])
        h = ctypes.c_void_p()
        _check(self.lib.tp_table_wrap_device(self.h, ctypes.byref(d), ptrs, nrows, ctypes.byref(h)))
        return Table(self, h, names)

    def plan(self, fact: "Table", dim: "Table | None", query: dict, agg_strategy=TP_AGG_AUTO,
             load_factor=0.0, expected_groups=0, join_partitions=0, lip=TP_LIP_AUTO,
             extra_dims=None) -> "Plan":
        """query: filter / join (many=True: repeated build keys, fan-out) / group /
        aggs as the oracle takes them, plus an
        optional dim_filter = dict(col=<dimension column>, lo=, hi=); a star join
        adds extra_joins = [dict(fact_col, dim_col, optional dim_filter)] over the
        tables extra_dims, their group fields on sides "dim1".."dim3"."""
        xjoins = query.get("extra_joins") or []
        extra_dims = list(extra_dims or [])
        if len(xjoins) != len(extra_dims):
            raise ValueError("one table in extra_dims per entry of extra_joins")
        d = tp_plan_desc()
        d.fact = fact.h
        d.dim = dim.h if dim is not None else None
        f = query.get("filter")
        d.filter = tp_filter(-1, 0, 0) if f is None else tp_filter(fact.col(f["col"]), f["lo"], f["hi"])
        j = query.get("join")
        d.join = tp_join(-1, -1) if j is None else tp_join(fact.col(j["fact_col"]), dim.col(j["dim_col"]))
        d.join_many = 1 if j is not None and j.get("many") else 0
        sides = {"fact": (TP_SIDE_FACT, fact), "dim": (TP_SIDE_DIM, dim)}
        for j, t in enumerate(extra_dims):
            sides[f"dim{j + 1}"] = (TP_SIDE_DIM + 1 + j, t)
        d.n_group = len(query["group"])
        for i, (side, col, bits) in enumerate(query["group"]):
            code, tab = sides[side]
            d.group[i] = tp_group_field(code, tab.col(col), bits)
        d.n_agg = len(query["aggs"])
        for i, ag in enumerate(query["aggs"]):
            if ag[0] == "sum":
                d.aggs[i] = tp_agg(TP_AGG_SUM, fact.col(ag[1]), -1, 0)
            elif ag[0] == "avg":
                d.aggs[i] = tp_agg(TP_AGG_AVG, fact.col(ag[1]), -1, 0)
            elif ag[0] == "count":
                d.aggs[i] = tp_agg(TP_AGG_COUNT, -1, -1, 0)
            elif ag[0] == "sum_mul_sub":
                d.aggs[i] = tp_agg(TP_AGG_SUM_MUL_SUB, fact.col(ag[1]), fact.col(ag[3]), ag[2])
            else:
                raise ValueError(ag)
        d.agg_strategy, d.load_factor, d.expected_groups = agg_strategy, load_factor, expected_groups
        d.join_partitions = join_partitions
        df = query.get("dim_filter")
        if df is not None:
            d.dim_filter, d.dim_filter_on = tp_filter(dim.col(df["col"]), df["lo"], df["hi"]), 1
        d.lip = lip
        d.n_extra_dims = len(xjoins)
        for j, (xj, t) in enumerate(zip(xjoins, extra_dims)):
            d.extra_dim[j] = t.h
            d.extra_join[j] = tp_join(fact.col(xj["fact_col"]), t.col(xj["dim_col"]))
            xf = xj.get("dim_filter")
            if xf is not None:
                d.extra_dim_filter[j], d.extra_dim_filter_on[j] = tp_filter(t.col(xf["col"]), xf["lo"], xf["hi"]), 1
        h = ctypes.c_void_p()
        _check(self.lib.tp_plan_create(self.h, ctypes.byref(d), ctypes.byref(h)))
        return Plan(self, h, list(query["aggs"]))


class Batch:
    """Many plans in one persistent, graph-captured launch (tp_batch_*)."""

    def __init__(self, eng: Engine, plans, tuning_path=None):
        self.eng, self.plans = eng, list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.h for p in self.plans])
        h = ctypes.c_void_p()
        tp = tuning_path.encode() if tuning_path else None
        _check(eng.lib.tp_batch_create(eng.h, arr, len(self.plans), tp, ctypes.byref(h)))
        self.h = h

    def execute(self) -> list:
        """Results in plan order; valid until the next execute() or destroy()."""
        out = (ctypes.c_void_p * len(self.plans))()
        _check(self.eng.lib.tp_batch_execute(self.h, out))
        return [Result(self.eng, ctypes.c_void_p(out[i]), p.aggs) for i, p in enumerate(self.plans)]

    @property
    def last_ms(self) -> float:
        return self.eng.lib.tp_batch_last_ms(self.h)

    def debug_stall(self, query: int, wait_ns: int = 0):
        """Makes query's finalisation wait for a tile that never comes (query
        -1 restores); the bounded wait gives up after wait_ns."""
        _check(self.eng.lib.tp_debug_batch_stall(self.h, query, wait_ns))

    def destroy(self):
        if self.h and self.eng.h:   # tp_shutdown already freed it otherwise
            self.eng.lib.tp_batch_destroy(self.h)
        self.h = None


class Server:
    """Request server (tp_server_*): submit plans, wait for results."""

    def __init__(self, eng: Engine, workers=4, max_inflight=0, cache_dims=True, batch=False):
        self.eng = eng
        h = ctypes.c_void_p()
        flags = (TP_SERVE_CACHE_DIM if cache_dims else 0) | (TP_SERVE_BATCH if batch else 0)
        _check(eng.lib.tp_server_start(eng.h, workers, max_inflight, flags, ctypes.byref(h)))
        self.h = h
        self._aggs = {}

    def submit(self, plan: "Plan") -> int:
        t = ctypes.c_uint64()
        _check(self.eng.lib.tp_submit(self.h, plan.h, ctypes.byref(t)))
        self._aggs[t.value] = plan.aggs
        return t.value

    def wait(self, ticket: int, timeout_s=None):
        """(Result, (submit_ns, start_ns, end_ns)); raises TPError on failure or timeout."""
        r = ctypes.c_void_p()
        times = (ctypes.c_int64 * 3)()
        ns = -1 if timeout_s is None else int(timeout_s * 1e9)
        code = self.eng.lib.tp_wait(self.h, ticket, ns, ctypes.byref(r), times)
        aggs = []
        if code not in (TP_TIMEOUT_CODE, TP_E_INVALID):   # the ticket is consumed
            aggs = self._aggs.pop(ticket, [])
        _check(code)
        return Result(self.eng, r, aggs), (times[0], times[1], times[2])

    def stats(self) -> dict:
        s = tp_server_stats()
        _check(self.eng.lib.tp_server_stats_get(self.h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in tp_server_stats._fields_}

    def stop(self):
        if self.h:
            self.eng.lib.tp_server_stop(self.h)
            self.h = None


TP_TIMEOUT_CODE = TP_E_TIMEOUT


def autotune(eng: Engine, plans, path: str):
    arr = (ctypes.c_void_p * len(plans))(*[p.h for p in plans])
    _check(eng.lib.tp_autotune(eng.h, arr, len(plans), path.encode()))


class Table:
    def __init__(self, eng: Engine, h, names):
        self.eng, self.h, self.names = eng, h, list(names)

    def col(self, name: str) -> int:
        return self.names.index(name)

    @property
    def rows(self) -> int:
        return self.eng.lib.tp_table_rows(self.h)

    @property
    def batches(self) -> int:
        return self.eng.lib.tp_table_batches(self.h)

    def place(self, placement: int):
        _check(self.eng.lib.tp_table_place(self.h, placement))

    def destroy(self):
        if self.h and self.eng.h:   # tp_shutdown already freed it otherwise
            self.eng.lib.tp_table_destroy(self.h)
        self.h = None


class Plan:
    def __init__(self, eng: Engine, h, aggs):
        self.eng, self.h, self.aggs = eng, h, aggs

    def execute(self) -> "Result":
        r = ctypes.c_void_p()
        _check(self.eng.lib.tp_execute(self.h, ctypes.byref(r)))
        return Result(self.eng, r, self.aggs)

    def destroy(self):
        if self.h and self.eng.h:   # tp_shutdown already freed it otherwise
            self.eng.lib.tp_plan_destroy(self.h)
        self.h = None


class Result:
    """Groups ascending by key; sums as (lo uint64, hi int64) pairs."""

    def __init__(self, eng: Engine, h, aggs):
        self.eng, self.h, self.aggs = eng, h, aggs

    @property
    def n_groups(self) -> int:
        return self.eng.lib.tp_result_groups(self.h)

    def _arr(self, ptr, dtype, n):
        if not ptr:
            raise TPError(TP_E_CUDA, last_error())
        return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(np.ctypeslib.as_ctypes_type(dtype))),
                                     shape=(max(n, 1),))[:n].copy()

    def keys(self) -> np.ndarray:
        return self._arr(self.eng.lib.tp_result_keys(self.h), np.uint64, self.n_groups)

    def counts(self) -> np.ndarray:
        return self._arr(self.eng.lib.tp_result_count(self.h), np.int64, self.n_groups)

    def sum_words(self, agg: int) -> np.ndarray:
        """[G, 2] uint64: low word, high word (two's complement)."""
        n = self.n_groups
        p = self.eng.lib.tp_result_sum(self.h, agg)
        if not p:
            raise TPError(TP_E_INVALID, last_error() or f"aggregate {agg} has no sum")
        raw = np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(ctypes.c_uint64)), shape=(max(n, 1) * 2,))
        return raw[: 2 * n].copy().reshape(n, 2)

    def avg(self, agg: int) -> np.ndarray:
        return self._arr(self.eng.lib.tp_result_avg(self.h, agg), np.float64, self.n_groups)

    def free(self):
        if self.h and self.eng.h:   # tp_shutdown already freed it otherwise
            self.eng.lib.tp_result_free(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.free()
