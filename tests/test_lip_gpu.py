"""Dimension predicates and lookahead information passing (Section 5): only
dimension rows that pass the predicate join; the lookahead (Bloom) filter of
their keys, tested on fact rows before the probe and before a partitioned join
spills them, must never change a result -- only the work done."""
import numpy as np
import pytest

import oracle
from datagen import workloads as W
from paper_2508_05029_gb300 import theseus as T
from tests.helpers import assert_matches_oracle
from tests.test_oracle_pins import _tiny

pytestmark = pytest.mark.gpu

LIPS = [T.TP_LIP_OFF, T.TP_LIP_AUTO, T.TP_LIP_ON]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_05029_gb300 import build
    build.build()


def _run(eng, fact, dim, q, placement=T.TP_DEVICE, **kw):
    ft = eng.table_from_numpy(fact, placement=placement)
    dt = eng.table_from_numpy(dim, placement=placement)
    p = eng.plan(ft, dt, q, **kw)
    try:
        return p.execute()
    finally:
        p.destroy()
        ft.destroy()
        dt.destroy()


@pytest.mark.parametrize("flags", [0, T.TP_FLAG_NO_JIT, T.TP_FLAG_NO_STAGED, T.TP_FLAG_NO_DIRECT_JOIN],
                         ids=["jit", "aot-staged", "plain", "hashed-join"])
@pytest.mark.parametrize("lip", LIPS, ids=["off", "auto", "on"])
def test_dim_predicate_device_tables(flags, lip):
    wl = W.config1(n_fact=400_003, n_dim=10_000)
    e = T.Engine(page_bytes=8 << 20, n_pages=64, batch_rows=1 << 20, flags=flags)
    try:
        for lo, hi in [(0, 4), (7, 7), (30, 40), (0, 24)]:
            q = dict(wl.query, dim_filter=dict(col="attr", lo=lo, hi=hi))
            f0 = e.stats()["lip_filters"]
            with _run(e, wl.fact, wl.dim, q, lip=lip) as r:
                assert_matches_oracle(r, oracle.run_query(wl.fact, wl.dim, q), q["aggs"])
            assert (e.stats()["lip_filters"] > f0) == (lip == T.TP_LIP_ON)   # auto: the table is small
    finally:
        e.close()


@pytest.mark.parametrize("lip", LIPS, ids=["off", "auto", "on"])
def test_dim_predicate_many_groups_and_pages(lip):
    """Paged tables (narrow pages), a dimension-side and a fact-side group
    field, a global aggregation; signed values, misses."""
    fact, dim = _tiny(30, 300_000, 20_000, 30_000, signed=True)
    q = dict(filter=dict(col="date", lo=100, hi=2400), join=dict(fact_col="fk", dim_col="pk"),
             group=[("dim", "attr", 5), ("fact", "qty", 14)],
             aggs=[("sum", "price"), ("count",), ("avg", "qty")],
             dim_filter=dict(col="attr", lo=3, hi=11))
    fact = dict(fact, qty=(fact["qty"] % 9000 + 9000) % 9000)
    ref = oracle.run_query(fact, dim, q)
    e = T.Engine(page_bytes=2 << 20, n_pages=128, batch_rows=65_536, flags=T.TP_FLAG_NO_DIRECT_JOIN)
    try:
        with _run(e, fact, dim, q, placement=T.TP_HOST_PAGES, lip=lip) as r:
            assert_matches_oracle(r, ref, q["aggs"])
    finally:
        e.close()


def test_dim_predicate_duplicates_only_among_admitted_rows():
    fact, dim = _tiny(31, 50_000, 400, 400)
    dim["pk"][5] = dim["pk"][6]
    dim["attr"][5], dim["attr"][6] = 1, 20
    e = T.Engine(page_bytes=8 << 20, n_pages=16, batch_rows=1 << 20)
    try:
        ok = dict(W.q_lowcard(), dim_filter=dict(col="attr", lo=10, hi=24))
        for flags_lip in LIPS:
            with _run(e, fact, dim, ok, lip=flags_lip) as r:
                assert_matches_oracle(r, oracle.run_query(fact, dim, ok), ok["aggs"])
        bad = dict(W.q_lowcard(), dim_filter=dict(col="attr", lo=0, hi=24))
        with pytest.raises(T.TPError) as err:
            _run(e, fact, dim, bad)
        assert err.value.status == "dup_key"
    finally:
        e.close()


def test_lip_partitioned_join_spills_less():
    """Hybrid hash join with a selective dimension predicate: with the
    lookahead filter, fact rows that cannot join are not spilled.  Budgets
    from roomy to tight; every run must match the oracle, and wherever rows
    spilled the filter must cut the spilled bytes."""
    n_dim, n_fact = 2_000_000, 3_000_007
    dim = W.config3_dim(n_dim=n_dim)
    fact = W.config3_fact(0, n_fact, n_dim=n_dim)
    q = dict(W.q_lowcard(), dim_filter=dict(col="attr", lo=0, hi=4))       # ~20% of the keys
    ref = oracle.run_query(fact, dim, q)
    spilled = 0
    for mb in (96, 80, 64, 56, 48):
        moved = {}
        for lip in (T.TP_LIP_OFF, T.TP_LIP_AUTO):
            e = T.Engine(page_bytes=2 << 20, n_pages=400, batch_rows=200_000)
            try:
                e.set_budget(mb << 20)
                d0, f0 = e.stats()["d2h_bytes"], e.stats()["lip_filters"]
                try:
                    r = _run(e, fact, dim, q, placement=T.TP_HOST_PAGES, join_partitions=16, lip=lip)
                except T.TPError as err:
                    assert err.status == "budget", err
                    continue
                with r:
                    assert_matches_oracle(r, ref, q["aggs"])
                st = e.stats()
                moved[lip] = st["d2h_bytes"] - d0
                assert (st["lip_filters"] > f0) == (lip == T.TP_LIP_AUTO)
                assert e.pages_free() == 400
            finally:
                e.close()
        print(f"budget {mb} MiB: spilled bytes without lookahead {moved.get(T.TP_LIP_OFF)}, "
              f"with {moved.get(T.TP_LIP_AUTO)}")
        if len(moved) < 2 or moved[T.TP_LIP_OFF] < (8 << 20):
            continue
        spilled += 1
        assert moved[T.TP_LIP_AUTO] < 0.6 * moved[T.TP_LIP_OFF]
    assert spilled >= 1


def test_dim_predicate_batched():
    wls = []
    for i, (lo, hi) in enumerate([(0, 4), (10, 24), (5, 5)]):
        wl = W.config1(n_fact=200_000 + i, n_dim=5_000)
        wl.query["dim_filter"] = dict(col="attr", lo=lo, hi=hi)
        wls.append(wl)
    e = T.Engine(page_bytes=8 << 20, n_pages=64, batch_rows=1 << 20)
    try:
        tabs, plans = [], []
        for wl in wls:
            ft = e.table_from_numpy(wl.fact, placement=T.TP_DEVICE)
            dt = e.table_from_numpy(wl.dim, placement=T.TP_DEVICE)
            tabs += [ft, dt]
            plans.append(e.plan(ft, dt, wl.query))
        b = T.Batch(e, plans)
        for wl, r in zip(wls, b.execute()):
            assert_matches_oracle(r, oracle.run(wl), wl.query["aggs"])
            r.free()
        b.destroy()
        for p in plans:
            p.destroy()
        for t in tabs:
            t.destroy()
    finally:
        e.close()


def test_dim_predicate_served_cache_keeps_predicates_apart():
    """Two plans over the same dimension with different predicates: the
    server's join-table cache must not hand one the other's table."""
    wl = W.config1(n_fact=300_000, n_dim=10_000)
    e = T.Engine(page_bytes=8 << 20, n_pages=64, batch_rows=1 << 20)
    try:
        ft = e.table_from_numpy(wl.fact, placement=T.TP_DEVICE)
        dt = e.table_from_numpy(wl.dim, placement=T.TP_DEVICE)
        qs = [dict(wl.query, dim_filter=dict(col="attr", lo=lo, hi=hi)) for lo, hi in [(0, 4), (5, 24), (0, 4)]]
        qs.append(dict(wl.query))
        plans = [e.plan(ft, dt, q) for q in qs]
        srv = T.Server(e, workers=2)
        try:
            for rep in range(2):
                tickets = [srv.submit(p) for p in plans]
                for q, t in zip(qs, tickets):
                    r, _ = srv.wait(t)
                    with r:
                        assert_matches_oracle(r, oracle.run_query(wl.fact, wl.dim, q), q["aggs"])
        finally:
            srv.stop()
        for p in plans:
            p.destroy()
        ft.destroy()
        dt.destroy()
    finally:
        e.close()


def test_invalid_dim_predicate():
    wl = W.config1(n_fact=1000, n_dim=100)
    e = T.Engine(page_bytes=8 << 20, n_pages=16, batch_rows=1 << 20)
    try:
        ft = e.table_from_numpy(wl.fact, placement=T.TP_DEVICE)
        dt = e.table_from_numpy(wl.dim, placement=T.TP_DEVICE)
        bad_mode = dict(wl.query, dim_filter=dict(col="attr", lo=0, hi=1))
        no_join = dict(filter=None, join=None, group=[], aggs=[("count",)], dim_filter=dict(col="attr", lo=0, hi=1))
        for q, kw in [(bad_mode, dict(lip=7)), (no_join, {})]:
            with pytest.raises(T.TPError) as err:
                e.plan(ft, dt, q, **kw)
            assert err.value.status == "invalid"
        ft.destroy()
        dt.destroy()
    finally:
        e.close()
