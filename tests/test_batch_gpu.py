"""Batched execution: many uneven queries in one persistent, graph-captured
launch, each result identical to the oracle's and to its own tp_execute."""
import os

import numpy as np
import pytest

import datagen
import oracle
from datagen import workloads as W
from paper_2508_05029_gb300 import theseus as T
from tests.helpers import assert_matches_oracle
from tests.test_oracle_pins import _tiny

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    from paper_2508_05029_gb300 import build
    build.build()
    e = T.Engine(page_bytes=8 << 20, n_pages=256, batch_rows=1 << 20)
    yield e
    e.close()


def _mix(n=10, scale=0.004):
    """Queries drawn like the batched workload, fact tables scaled down."""
    sz = W.config4_sizes(n_queries=n, fact_hi=5_000_000, dim_hi=200_000)
    out = []
    for q in range(n):
        out.append(W.config4_query(q, int(sz["fact"][q]), int(sz["dim"][q]), int(sz["cutoff"][q]),
                                   int(sz["groups"][q]), fact_scale=scale))
    return out


def _device_plans(eng, wls, **kw):
    tabs, plans = [], []
    for wl in wls:
        ft = eng.table_from_numpy(wl.fact, placement=T.TP_DEVICE)
        dt = eng.table_from_numpy(wl.dim, placement=T.TP_DEVICE) if wl.dim is not None else None
        tabs += [ft] + ([dt] if dt is not None else [])
        plans.append(eng.plan(ft, dt, wl.query, **kw))
    return tabs, plans


@pytest.mark.parametrize("flags", [0, T.TP_FLAG_NO_JIT])
def test_batch_matches_oracle_and_replays(flags):
    wls = _mix()
    wls.append(W.config1(n_fact=300_007))                       # 8-bit key: shared-memory tables
    fact, dim = _tiny(3, 5000, 300, 400, signed=True)         # misses, signed values
    wls.append(W.Workload("tiny", fact, dim, W.q_lowcard()))
    eng = T.Engine(page_bytes=8 << 20, n_pages=256, batch_rows=1 << 20, flags=flags)
    try:
        tabs, plans = _device_plans(eng, wls)
        refs = [oracle.run(wl) for wl in wls]
        b = T.Batch(eng, plans)
        for rep in range(2):                                        # graph replay gives the same answers
            res = b.execute()
            for wl, ref, r in zip(wls, refs, res):
                assert_matches_oracle(r, ref, wl.query["aggs"])
                r.free()
        assert b.last_ms > 0
        assert (eng.stats()["jit_launches"] > 0) == (flags == 0)
        b.destroy()
        for p in plans:
            p.destroy()
        for t in tabs:
            t.destroy()
    finally:
        eng.close()


@pytest.mark.parametrize("flags", [0, T.TP_FLAG_NO_JIT])
def test_batch_exact_and_hash_paths(flags):
    """Sums that need 128 bits, and hashed (not direct-mapped) join keys; the
    run-time compiled and the ahead-of-time queue kernels."""
    e = T.Engine(page_bytes=8 << 20, n_pages=64, batch_rows=1 << 20, flags=T.TP_FLAG_NO_DIRECT_JOIN | flags)
    try:
        n = 20_000
        big = dict(a=np.full(n, (1 << 62) + 7, np.int64), b=np.full(n, -(1 << 62), np.int64),
                   fk=datagen.uniform(9, 1, np.int32, n, 0, 99), d=datagen.uniform(9, 2, np.int32, n, 0, 9))
        dim = dict(pk=np.arange(100, dtype=np.int32), attr=(np.arange(100) % 7).astype(np.int32))
        qb = dict(filter=dict(col="d", lo=1, hi=8), join=dict(fact_col="fk", dim_col="pk"),
                  group=[("dim", "attr", 3)], aggs=[("sum_mul_sub", "a", 1 << 62, "b"), ("avg", "b"), ("count",)])
        wls = [W.Workload("big", big, dim, qb)] + _mix(4)
        tabs, plans = _device_plans(e, wls)
        b = T.Batch(e, plans)
        j0 = e.stats()["jit_launches"]
        for wl, r in zip(wls, b.execute()):
            assert_matches_oracle(r, oracle.run(wl), wl.query["aggs"])
        assert (e.stats()["jit_launches"] > j0) == (flags == 0)
        assert e.stats()["jit_failures"] == 0
        b.destroy()
        for p in plans:
            p.destroy()
        for t in tabs:
            t.destroy()
    finally:
        e.close()


def test_batch_rejections(eng):
    wl = W.config1(n_fact=10_000, n_dim=1_000)
    dt = eng.table_from_numpy(wl.dim, placement=T.TP_DEVICE)
    fd = eng.table_from_numpy(wl.fact, placement=T.TP_DEVICE)
    wide = dict(wl.query, group=[("fact", "qty", 21)])
    p = eng.plan(fd, dt, wide)
    with pytest.raises(T.TPError) as e:
        T.Batch(eng, [p])
    assert e.value.status == "invalid"
    p.destroy()
    bad = {k: v.copy() for k, v in wl.dim.items()}
    bad["pk"][3] = bad["pk"][4]
    dbad = eng.table_from_numpy(bad, placement=T.TP_DEVICE)
    p = eng.plan(fd, dbad, wl.query)
    b = T.Batch(eng, [p])
    with pytest.raises(T.TPError) as e:
        b.execute()
    assert e.value.status == "dup_key"
    b.destroy()
    p.destroy()
    for t in (dt, fd, dbad):
        t.destroy()


def test_autotune_table_roundtrip(eng, tmp_path):
    wls = _mix(6)
    tabs, plans = _device_plans(eng, wls)
    path = str(tmp_path / "tune.txt")
    T.autotune(eng, plans, path)
    lines = [l for l in open(path) if not l.startswith("#")]
    assert len(lines) >= 1
    b = T.Batch(eng, plans, tuning_path=path)
    for wl, r in zip(wls, b.execute()):
        assert_matches_oracle(r, oracle.run(wl), wl.query["aggs"])
    b.destroy()
    for p in plans:
        p.destroy()
    for t in tabs:
        t.destroy()


def test_bounded_wait_times_out_and_context_survives(eng):
    """A dependency that is never published: the persistent kernel's bounded
    wait gives up, the host reports TP_E_TIMEOUT, and the same batch (and
    device context) runs correctly afterwards."""
    wls = _mix(n=4)
    tabs, plans = _device_plans(eng, wls)
    refs = [oracle.run(wl) for wl in wls]
    b = T.Batch(eng, plans)
    try:
        b.debug_stall(2, wait_ns=20_000_000)       # query 2 waits for a tile that never comes; 20 ms limit
        with pytest.raises(T.TPError) as err:
            b.execute()
        assert err.value.status == "timeout"
        b.debug_stall(-1)
        for wl, ref, r in zip(wls, refs, b.execute()):
            assert_matches_oracle(r, ref, wl.query["aggs"])
            r.free()
    finally:
        b.destroy()
        for p in plans:
            p.destroy()
        for t in tabs:
            t.destroy()
