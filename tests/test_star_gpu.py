"""Star joins: further dimension tables, each joined on its own fact foreign
key (with its own predicate and lookahead filter); results identical to the
oracle's on every kernel path, table placement and join kind."""
import numpy as np
import pytest

import oracle
from datagen import workloads as W
from paper_2508_05029_gb300 import theseus as T
from tests.helpers import assert_matches_oracle
from tests.test_oracle_pins import _star_query, _star_tiny

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_05029_gb300 import build
    build.build()


def _narrow_keys(fact, extra):
    """int32 foreign and primary keys (small stages: the run-time compiled kernel)."""
    fact = dict(fact)
    for j in range(len(extra)):
        fact[f"fk{j + 2}"] = fact[f"fk{j + 2}"].astype(np.int32)
    return fact, [dict(x, pk=x["pk"].astype(np.int32)) for x in extra]


def _run(eng, fact, dim, extra, q, placement=T.TP_DEVICE, **kw):
    ft = eng.table_from_numpy(fact, placement=placement)
    dt = eng.table_from_numpy(dim, placement=placement)
    xt = [eng.table_from_numpy(x, placement=placement) for x in extra]
    p = eng.plan(ft, dt, q, extra_dims=xt, **kw)
    try:
        return p.execute()
    finally:
        p.destroy()
        for t in [ft, dt] + xt:
            t.destroy()


@pytest.mark.parametrize("flags", [0, T.TP_FLAG_NO_JIT, T.TP_FLAG_NO_STAGED, T.TP_FLAG_NO_DIRECT_JOIN],
                         ids=["jit", "no-jit", "plain", "hashed-joins"])
@pytest.mark.parametrize("n_extra", [1, 2, 3])
def test_star_join_matches_oracle(flags, n_extra):
    fact, dim, extra = _star_tiny(50 + n_extra, 400_003, [20_000, 5_000, 3_000, 1_000][:n_extra + 1],
                                  [24_000, 6_000, 3_500, 1_200][:n_extra + 1])
    fact, extra = _narrow_keys(fact, extra)
    filters = [(None, None, None, None),
               (dict(col="attr", lo=0, hi=20), dict(col="attr", lo=3, hi=24), dict(col="band", lo=0, hi=2),
                dict(col="attr", lo=0, hi=12))]
    e = T.Engine(page_bytes=8 << 20, n_pages=64, batch_rows=1 << 20, flags=flags)
    try:
        for flt in filters:
            q = _star_query(n_extra, flt)
            j0 = e.stats()["jit_launches"]
            with _run(e, fact, dim, extra, q) as r:
                assert_matches_oracle(r, oracle.run_query(fact, dim, q, extra), q["aggs"])
            if flags == 0 and n_extra == 1:
                assert e.stats()["jit_launches"] > j0      # the star shape ran compiled for itself
    finally:
        e.close()


@pytest.mark.parametrize("lip", [T.TP_LIP_OFF, T.TP_LIP_ON], ids=["lip-off", "lip-on"])
def test_star_join_lookahead_and_wide_keys(lip):
    """int64 sparse keys in the further tables (hashed), predicates on each,
    lookahead filters forced on: one per filtered dimension."""
    fact, dim, extra = _star_tiny(60, 300_001, [10_000, 8_000, 6_000], [12_000, 9_000, 7_000])
    # an odd multiplier modulo 2^64 is a bijection: unique sparse keys, misses stay misses
    scramble = lambda v: (v.astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)).view(np.int64)
    for j, x in enumerate(extra):
        x["pk"] = scramble(x["pk"])
        fact[f"fk{j + 2}"] = scramble(fact[f"fk{j + 2}"])
    q = _star_query(2, (dict(col="attr", lo=0, hi=9), dict(col="band", lo=1, hi=3), dict(col="attr", lo=5, hi=24)))
    e = T.Engine(page_bytes=8 << 20, n_pages=64, batch_rows=1 << 20)
    try:
        f0 = e.stats()["lip_filters"]
        with _run(e, fact, dim, extra, q, lip=lip) as r:
            assert_matches_oracle(r, oracle.run_query(fact, dim, q, extra), q["aggs"])
        assert e.stats()["lip_filters"] - f0 == (3 if lip == T.TP_LIP_ON else 0)
    finally:
        e.close()


def test_star_join_many_groups_and_pages():
    """Global aggregation (a wide fact-side field), every table in host pages."""
    fact, dim, extra = _star_tiny(61, 250_000, [9_000, 4_000], [10_000, 4_500])
    fact["okey"] = (np.arange(250_000, dtype=np.int64) * 7919) % 60_013
    q = _star_query(1, (None, dict(col="attr", lo=2, hi=22)))
    q["group"] = [("fact", "okey", 20), ("dim1", "band", 2), ("dim", "attr", 5)]
    ref = oracle.run_query(fact, dim, q, extra)
    for flags in (0, T.TP_FLAG_NO_DIRECT_AGG):
        e = T.Engine(page_bytes=2 << 20, n_pages=256, batch_rows=65_536, flags=flags)
        try:
            with _run(e, fact, dim, extra, q, placement=T.TP_HOST_PAGES) as r:
                assert_matches_oracle(r, ref, q["aggs"])
        finally:
            e.close()


def test_star_join_partitioned_first_join():
    """The first join runs partitioned and spills; the further table stays
    resident and is probed in both phases."""
    n_dim, n_fact = 2_000_000, 2_000_003
    dim = W.config3_dim(n_dim=n_dim)
    fact = W.config3_fact(0, n_fact, n_dim=n_dim)
    extra = [dict(pk=np.arange(3000, dtype=np.int32), band=(np.arange(3000) % 4).astype(np.uint8),
                  attr=(np.arange(3000) % 25).astype(np.int32))]
    fact["fk2"] = ((np.arange(n_fact, dtype=np.int64) * 2654435761) % 3500).astype(np.int32)
    q = dict(W.q_lowcard(), extra_joins=[dict(fact_col="fk2", dim_col="pk", dim_filter=dict(col="attr", lo=0, hi=19))])
    q["group"] = [("fact", "flag", 2), ("dim", "attr", 5), ("dim1", "band", 2)]
    ref = oracle.run_query(fact, dim, q, extra)
    e = T.Engine(page_bytes=2 << 20, n_pages=400, batch_rows=200_000)
    try:
        e.set_budget(96 << 20)
        d0 = e.stats()["d2h_bytes"]
        with _run(e, fact, dim, extra, q, placement=T.TP_HOST_PAGES, join_partitions=16) as r:
            assert_matches_oracle(r, ref, q["aggs"])
        assert e.stats()["d2h_bytes"] - d0 > 8 << 20          # partitions spilled
        assert e.pages_free() == 400
    finally:
        e.close()


def test_star_join_errors_and_served():
    fact, dim, extra = _star_tiny(62, 50_000, [2_000, 800], [2_200, 900])
    fact, extra = _narrow_keys(fact, extra)
    q = _star_query(1)
    e = T.Engine(page_bytes=8 << 20, n_pages=64, batch_rows=1 << 20)
    try:
        ft = e.table_from_numpy(fact, placement=T.TP_DEVICE)
        dt = e.table_from_numpy(dim, placement=T.TP_DEVICE)
        xt = e.table_from_numpy(extra[0], placement=T.TP_DEVICE)
        p = e.plan(ft, dt, q, extra_dims=[xt])
        # batched execution takes one dimension
        with pytest.raises(T.TPError) as err:
            T.Batch(e, [p])
        assert err.value.status == "invalid"
        # the server runs star plans (the first table cached, the further one built per request)
        srv = T.Server(e, workers=2)
        try:
            ref = oracle.run_query(fact, dim, q, extra)
            for t in [srv.submit(p) for _ in range(4)]:
                r, _ = srv.wait(t)
                with r:
                    assert_matches_oracle(r, ref, q["aggs"])
        finally:
            srv.stop()
        p.destroy()
        # a duplicate key in a further dimension, and a field outside its width
        bad = dict(extra[0], pk=extra[0]["pk"].copy())
        bad["pk"][7] = bad["pk"][8]
        bt = e.table_from_numpy(bad, placement=T.TP_DEVICE)
        p = e.plan(ft, dt, q, extra_dims=[bt])
        with pytest.raises(T.TPError) as err:
            p.execute()
        assert err.value.status == "dup_key"
        p.destroy()
        wide = dict(q, group=[("dim", "attr", 5), ("dim1", "attr", 3)])     # attr up to 24 needs 5 bits
        p = e.plan(ft, dt, wide, extra_dims=[xt])
        with pytest.raises(T.TPError) as err:
            p.execute()
        assert err.value.status == "range"
        p.destroy()
        for t in (ft, dt, xt, bt):
            t.destroy()
    finally:
        e.close()
