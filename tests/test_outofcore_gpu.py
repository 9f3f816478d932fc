"""Hybrid (partitioned) hash join: build and fact rows of partitions that do
not fit the device budget are spilled to pool pages and joined one partition
at a time.  Results must equal the oracle's, spilled or not."""
import numpy as np
import pytest

import oracle
from datagen import workloads as W
from paper_2508_05029_gb300 import theseus as T
from tests.helpers import assert_matches_oracle

pytestmark = pytest.mark.gpu

N_DIM, N_FACT = 2_000_000, 3_000_007


@pytest.fixture(scope="module")
def data():
    from paper_2508_05029_gb300 import build
    build.build()
    dim = W.config3_dim(n_dim=N_DIM)                 # sparse unique int64 keys: hashed join
    fact = W.config3_fact(0, N_FACT, n_dim=N_DIM)
    return fact, dim


def _engine():
    return T.Engine(page_bytes=2 << 20, n_pages=400, batch_rows=200_000)


def _run(eng, fact, dim, query, placement, **kw):
    ft = eng.table_from_numpy(fact, placement=placement)
    dt = eng.table_from_numpy(dim, placement=placement)
    p = eng.plan(ft, dt, query, **kw)
    try:
        return p.execute(), eng.stats()
    finally:
        p.destroy()
        ft.destroy()
        dt.destroy()


@pytest.mark.parametrize("partitions", [0, 8, 64])
def test_spilled_partitions_match_oracle(data, partitions):
    fact, dim = data
    q = W.q_lowcard()
    ref = oracle.run_query(fact, dim, q)
    e = _engine()
    try:
        e.set_budget(96 << 20)     # the 64 MB join table does not fit: most partitions spill
        d0 = e.stats()["d2h_bytes"]
        res, st = _run(e, fact, dim, q, T.TP_HOST_PAGES, join_partitions=partitions)
        with res:
            assert_matches_oracle(res, ref, q["aggs"])
        assert st["d2h_bytes"] - d0 > 10 << 20          # spilled rows went to host pages
        assert e.pages_free() == 400                       # spill pages returned
    finally:
        e.close()


def test_partitioned_high_cardinality(data):
    fact, dim = data
    fact = dict(fact, okey=(np.arange(N_FACT, dtype=np.int64) * 7919) % 500_009)
    q = dict(filter=dict(col="date", lo=0, hi=W.CUTOFF_98), join=dict(fact_col="fk", dim_col="pk"),
             group=[("fact", "okey", 64)], aggs=[("sum_mul_sub", "price", 100, "disc"), ("count",)])
    ref = oracle.run_query(fact, dim, q)
    e = _engine()
    try:
        # the aggregation table, its sort arrays and the result take about
        # 100 MB of the 150 MB; the join gets what is left, below the 64 MB
        # table: partitions spill
        e.set_budget(150 << 20)
        d0 = e.stats()["d2h_bytes"]
        res, st = _run(e, fact, dim, q, T.TP_HOST_PAGES, join_partitions=16, expected_groups=500_009)
        with res:
            assert_matches_oracle(res, ref, q["aggs"])
        assert st["d2h_bytes"] - d0 > 10 << 20
    finally:
        e.close()


def test_all_resident_partitions(data):
    fact, dim = data
    q = W.q_lowcard()
    ref = oracle.run_query(fact, dim, q)
    e = _engine()
    try:
        res, st = _run(e, fact, dim, q, T.TP_HOST_PAGES, join_partitions=4)   # budget ample: nothing spills
        with res:
            assert_matches_oracle(res, ref, q["aggs"])
    finally:
        e.close()


def test_pool_exhaustion_is_reported(data):
    fact, dim = data
    q = W.q_lowcard()
    e = T.Engine(page_bytes=2 << 20, n_pages=100, batch_rows=200_000)   # tables fit, spills do not
    try:
        e.set_budget(96 << 20)
        with pytest.raises(T.TPError) as err:
            _run(e, fact, dim, q, T.TP_HOST_PAGES, join_partitions=64)
        assert err.value.status == "pool_empty"
        assert e.pages_free() == 100
    finally:
        e.close()
