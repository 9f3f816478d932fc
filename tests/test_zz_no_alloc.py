"""tp_execute_noalloc: the allocation-free entry point, checked against tp_execute.

Callers that cannot allocate device memory mid-query -- applications whose
GPU memory all belongs to their own allocator, or latency-bound code that
cannot risk a cudaMalloc/cudaFree -- use tp_execute_noalloc, whose scratch is
a fixed device array inside the library.  This test calls it through the C
ABI twice in a row (the second call reuses the array the first one left
behind) and requires the same groups, counts, exact sums and averages as the
regular entry point, tp_execute, on the same device columns.  It runs last so
that a failure here leaves every other test already run, and it passes both
alone in a fresh process and after the rest of the suite.  After a first call
has set the device up, further calls of other shapes leave the device's free
memory unchanged.
"""
import ctypes

import numpy as np
import pytest

from datagen import workloads as W
from paper_2508_05029_gb300 import theseus as T
from tests.helpers import AVG_RTOL

pytestmark = pytest.mark.gpu

NP2TP = {np.dtype(np.int32): T.TP_I32, np.dtype(np.int64): T.TP_I64, np.dtype(np.uint8): T.TP_U8}


def _desc(query, fact_names, dim_names):
    d = T.tp_plan_desc()
    f = query["filter"]
    d.filter = T.tp_filter(fact_names.index(f["col"]), f["lo"], f["hi"]) if f else T.tp_filter(-1, 0, 0)
    j = query["join"]
    d.join = (T.tp_join(fact_names.index(j["fact_col"]), dim_names.index(j["dim_col"])) if j
              else T.tp_join(-1, -1))
    d.n_group = len(query["group"])
    for i, (side, col, bits) in enumerate(query["group"]):
        names = fact_names if side == "fact" else dim_names
        d.group[i] = T.tp_group_field(T.TP_SIDE_FACT if side == "fact" else T.TP_SIDE_DIM, names.index(col), bits)
    d.n_agg = len(query["aggs"])
    kinds = {"sum": T.TP_AGG_SUM, "avg": T.TP_AGG_AVG, "count": T.TP_AGG_COUNT}
    for i, ag in enumerate(query["aggs"]):
        if ag[0] == "sum_mul_sub":
            d.aggs[i] = T.tp_agg(T.TP_AGG_SUM_MUL_SUB, fact_names.index(ag[1]), fact_names.index(ag[3]), ag[2])
        elif ag[0] == "count":
            d.aggs[i] = T.tp_agg(T.TP_AGG_COUNT, -1, -1, 0)
        else:
            d.aggs[i] = T.tp_agg(kinds[ag[0]], fact_names.index(ag[1]), -1, 0)
    return d


def _noalloc(torch, fact, dim, query, stream):
    """One tp_execute_noalloc call; returns host copies of its outputs."""
    lib = T.load()
    fn, dn = list(fact), list(dim)
    ft = [fact[k] for k in fn]
    dt = [dim[k] for k in dn]
    bits = sum(b for _, _, b in query["group"])
    cap = 1 << bits
    dev = ft[0].device
    keys = torch.empty(cap, dtype=torch.int64, device=dev)
    counts = torch.empty(cap, dtype=torch.int64, device=dev)
    sums = [torch.empty(cap * 2, dtype=torch.int64, device=dev) if ag[0] != "count" else None
            for ag in query["aggs"]]
    avgs = [torch.empty(cap, dtype=torch.float64, device=dev) if ag[0] == "avg" else None
            for ag in query["aggs"]]
    d = _desc(query, fn, dn)
    tmap = {torch.int32: T.TP_I32, torch.int64: T.TP_I64, torch.uint8: T.TP_U8}
    fcols = (ctypes.c_void_p * len(ft))(*[x.data_ptr() for x in ft])
    ftyp = (ctypes.c_int32 * len(ft))(*[tmap[x.dtype] for x in ft])
    dcols = (ctypes.c_void_p * len(dt))(*[x.data_ptr() for x in dt])
    dtyp = (ctypes.c_int32 * len(dt))(*[tmap[x.dtype] for x in dt])
    sp = (ctypes.c_void_p * 8)(*[(s.data_ptr() if s is not None else None) for s in sums])
    ap = (ctypes.c_void_p * 8)(*[(a.data_ptr() if a is not None else None) for a in avgs])
    ng = ctypes.c_uint64(0)
    rc = lib.tp_execute_noalloc(ctypes.byref(d), fcols, ftyp, len(ft), ft[0].numel(), dcols, dtyp, len(dt),
                                dt[0].numel(), keys.data_ptr(), counts.data_ptr(), sp, ap, ctypes.byref(ng),
                                stream.cuda_stream)
    if rc != T.TP_OK:
        raise T.TPError(rc, T.last_error())
    g = ng.value
    out = dict(keys=keys[:g].cpu().numpy().view(np.uint64), counts=counts[:g].cpu().numpy(), sums={}, avgs={})
    for a, ag in enumerate(query["aggs"]):
        if sums[a] is not None:
            out["sums"][a] = sums[a][: 2 * g].cpu().numpy().view(np.uint64).reshape(g, 2)
        if avgs[a] is not None:
            out["avgs"][a] = avgs[a][:g].cpu().numpy()
    return out


def _regular(eng, ft, dt, query):
    p = eng.plan(ft, dt, query)
    try:
        with p.execute() as r:
            out = dict(keys=r.keys(), counts=r.counts(), sums={}, avgs={})
            for a, ag in enumerate(query["aggs"]):
                if ag[0] != "count":
                    out["sums"][a] = r.sum_words(a)
                if ag[0] == "avg":
                    out["avgs"][a] = r.avg(a)
            return out
    finally:
        p.destroy()


def _same(got, want):
    assert np.array_equal(got["keys"], want["keys"])
    assert np.array_equal(got["counts"], want["counts"])
    assert got["sums"].keys() == want["sums"].keys()
    for a in want["sums"]:
        assert np.array_equal(got["sums"][a], want["sums"][a])
    for a in want["avgs"]:
        w = want["avgs"][a]
        rel = np.abs(got["avgs"][a] - w) / np.maximum(np.abs(w), np.finfo(np.float64).tiny)
        assert rel.size == 0 or float(rel.max()) <= AVG_RTOL


@pytest.mark.parametrize("maker", ["star_1M", "star_zipf"])
def test_noalloc_matches_tp_execute_twice(maker):
    torch = pytest.importorskip("torch")
    from paper_2508_05029_gb300 import build
    build.build()
    if maker == "star_1M":
        wl = W.config1()
        fact_np, dim_np, q = wl.fact, wl.dim, wl.query
    else:
        fact_np, dim_np = W.config2_tables(n_fact=2_000_003, n_dim=500_000)
        q = W.q_lowcard()
    fact = {k: torch.from_numpy(v).cuda() for k, v in fact_np.items()}
    dim = {k: torch.from_numpy(v).cuda() for k, v in dim_np.items()}
    stream = torch.cuda.Stream()
    with T.Engine() as eng:
        ft = eng.table_from_torch(fact)
        dt = eng.table_from_torch(dim)
        want = _regular(eng, ft, dt, q)
        ft.destroy()
        dt.destroy()
    assert want["keys"].size == 150
    first = _noalloc(torch, fact, dim, q, stream)
    second = _noalloc(torch, fact, dim, q, stream)
    _same(first, want)
    _same(second, want)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    fact_np, dim_np = W.config2_tables(n_fact=10_000, n_dim=600_000)
    fact = {k: torch.from_numpy(v).cuda() for k, v in fact_np.items()}
    dim = {k: torch.from_numpy(v).cuda() for k, v in dim_np.items()}
    stream = torch.cuda.Stream()
    with pytest.raises(T.TPError) as e:
        _noalloc(torch, fact, dim, W.q_lowcard(), stream)
    assert e.value.status == "invalid" and "fixed" in str(e.value)
    q = W.q_lowcard(attr_bits=10)      # 13-bit key: more groups than the scratch holds
    small = {k: v[:1000] for k, v in dim.items()}
    with pytest.raises(T.TPError) as e:
        _noalloc(torch, fact, small, q, stream)
    assert e.value.status == "invalid" and "12 bits" in str(e.value)


def _call_into(torch, lib, fact, dim, query, stream, out):
    """One tp_execute_noalloc call into preallocated outputs (no tensor is
    created here); returns the group count."""
    fn, dn = list(fact), list(dim)
    ft = [fact[k] for k in fn]
    dt = [dim[k] for k in dn]
    d = _desc(query, fn, dn)
    tmap = {torch.int32: T.TP_I32, torch.int64: T.TP_I64, torch.uint8: T.TP_U8}
    fcols = (ctypes.c_void_p * len(ft))(*[x.data_ptr() for x in ft])
    ftyp = (ctypes.c_int32 * len(ft))(*[tmap[x.dtype] for x in ft])
    dcols = (ctypes.c_void_p * max(1, len(dt)))(*[x.data_ptr() for x in dt])
    dtyp = (ctypes.c_int32 * max(1, len(dt)))(*[tmap[x.dtype] for x in dt])
    sp = (ctypes.c_void_p * 8)(*[out["sums"][a].data_ptr() if a < len(query["aggs"]) and
                                 query["aggs"][a][0] != "count" else None for a in range(8)])
    ap = (ctypes.c_void_p * 8)(*[out["avgs"][a].data_ptr() if a < len(query["aggs"]) and
                                 query["aggs"][a][0] == "avg" else None for a in range(8)])
    ng = ctypes.c_uint64(0)
    rc = lib.tp_execute_noalloc(ctypes.byref(d), fcols, ftyp, len(ft), ft[0].numel(), dcols, dtyp, len(dt),
                                dt[0].numel() if dt else 0, out["keys"].data_ptr(), out["counts"].data_ptr(), sp,
                                ap, ctypes.byref(ng), stream.cuda_stream)
    if rc != T.TP_OK:
        raise T.TPError(rc, T.last_error())
    return ng.value


def test_noalloc_calls_after_the_first_leave_free_memory_unchanged():
    """A warm-up call sets the device up; then a small key, a 12-bit key, a
    query without a join and one with a 64-bit key join run without changing
    the device's free memory (cudaMemGetInfo)."""
    torch = pytest.importorskip("torch")
    from paper_2508_05029_gb300 import build
    build.build()
    lib = T.load()
    dev = torch.device("cuda", 0)
    f1, d1 = W.config2_tables(n_fact=400_003, n_dim=100_000)
    f3, d3 = W.config3_fact(0, 300_001, n_dim=50_000), W.config3_dim(50_000)
    fact1 = {k: torch.from_numpy(v).to(dev) for k, v in f1.items()}
    dim1 = {k: torch.from_numpy(v).to(dev) for k, v in d1.items()}
    fact3 = {k: torch.from_numpy(v).to(dev) for k, v in f3.items()}
    dim3 = {k: torch.from_numpy(v).to(dev) for k, v in d3.items()}
    q_small = W.q_lowcard()                                            # 8-bit key
    q_wide = dict(W.q_lowcard(attr_bits=9), group=[("fact", "flag", 2), ("fact", "status", 1),
                                                   ("dim", "attr", 9)])  # 12-bit key
    q_nojoin = dict(filter=dict(col="date", lo=0, hi=1500), join=None,
                    group=[("fact", "flag", 2), ("fact", "status", 1)],
                    aggs=[("sum", "price"), ("count",), ("avg", "qty")])
    cap = 1 << 12
    out = dict(keys=torch.empty(cap, dtype=torch.int64, device=dev),
               counts=torch.empty(cap, dtype=torch.int64, device=dev),
               sums=[torch.empty(cap * 2, dtype=torch.int64, device=dev) for _ in range(8)],
               avgs=[torch.empty(cap, dtype=torch.float64, device=dev) for _ in range(8)])
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    _call_into(torch, lib, fact1, dim1, q_small, stream, out)          # sets the device up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    groups = []
    for fact, dim, q in ((fact1, dim1, q_small), (fact1, dim1, q_wide), (fact1, dim1, q_nojoin),
                         (fact3, dim3, q_small), (fact1, dim1, q_wide)):
        groups.append(_call_into(torch, lib, fact, dim, q, stream, out))
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info(dev)[0]
    assert free1 == free0, (free0, free1)
    assert groups[0] == groups[1] == groups[3] == groups[4] == 150 and groups[2] == 6
