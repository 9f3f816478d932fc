"""Join fan-out: the first join's build keys repeat, a fact row pairs with every
admitted dimension row holding its key, and every pair counts once.  Results
identical to the oracle's on every kernel path and table placement."""
import numpy as np
import pytest

import datagen
import oracle
from datagen import workloads as W
from paper_2508_05029_gb300 import theseus as T
from tests.helpers import assert_matches_oracle
from tests.test_oracle_pins import _star_tiny, _tiny

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_05029_gb300 import build
    build.build()


def _fanout_tables(seed, n_fact, n_keys, span, sparse=False):
    """Key k appears 1 + (k mod 4) times among the dimension rows (shuffled);
    fact keys drawn from a wider span, so some rows miss."""
    fact, _ = _tiny(seed, n_fact, 0, span)
    reps = 1 + np.arange(n_keys) % 4
    pk = np.repeat(np.arange(n_keys, dtype=np.int64), reps)
    perm = datagen.fill(5000 + seed, 1, datagen.PERM, np.int64, len(pk), b=len(pk))
    dim = dict(pk=pk[perm].astype(np.int32), attr=datagen.uniform(5000 + seed, 2, np.int32, len(pk), 0, 24))
    if sparse:   # int64 keys through an odd multiplier mod 2^64: hashed 64-bit tables
        mul = np.uint64(0x9E3779B97F4A7C15)
        dim["pk"] = (dim["pk"].astype(np.uint64) * mul).view(np.int64)
        fact["fk"] = (fact["fk"].astype(np.uint64) * mul).view(np.int64)
    return fact, dim


def _run(eng, fact, dim, q, placement=T.TP_DEVICE, extra=(), **kw):
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


def _fanout_query(dflt=None):
    return dict(W.q_lowcard(), join=dict(fact_col="fk", dim_col="pk", many=True), dim_filter=dflt)


@pytest.mark.parametrize("flags", [0, T.TP_FLAG_NO_JIT, T.TP_FLAG_NO_STAGED, T.TP_FLAG_NO_DIRECT_JOIN],
                         ids=["jit", "no-jit", "plain", "hashed-join"])
@pytest.mark.parametrize("sparse", [False, True], ids=["dense-keys", "sparse-int64-keys"])
def test_fanout_matches_oracle(flags, sparse):
    fact, dim = _fanout_tables(80 + sparse, 400_003, 20_000, 24_000, sparse=sparse)
    e = T.Engine(page_bytes=8 << 20, n_pages=64, batch_rows=1 << 20, flags=flags)
    try:
        for dflt, lip in [(None, T.TP_LIP_AUTO), (dict(col="attr", lo=3, hi=14), T.TP_LIP_ON),
                          (dict(col="attr", lo=3, hi=14), T.TP_LIP_OFF)]:
            q = _fanout_query(dflt)
            j0 = e.stats()["jit_launches"]
            with _run(e, fact, dim, q, lip=lip) as r:
                assert_matches_oracle(r, oracle.run_query(fact, dim, q), q["aggs"])
            if flags == 0:
                assert e.stats()["jit_launches"] > j0
    finally:
        e.close()


def test_fanout_many_groups_pages_and_star():
    """Global aggregation over a fact-side order key and the dimension
    attribute, paged tables, and a further (unique-key) dimension."""
    fact, dim = _fanout_tables(82, 250_000, 9_000, 10_000)
    _, _, extra = _star_tiny(82, 250_000, [9_000, 3_000], [10_000, 3_300])
    fact["fk2"] = datagen.uniform(5082, 7, np.int64, 250_000, 0, 3_299)
    fact["okey"] = (np.arange(250_000, dtype=np.int64) * 7919) % 40_009
    q = _fanout_query(dict(col="attr", lo=0, hi=20))
    q["extra_joins"] = [dict(fact_col="fk2", dim_col="pk", dim_filter=dict(col="band", lo=0, hi=2))]
    q["group"] = [("fact", "okey", 16), ("dim", "attr", 5), ("dim1", "band", 2)]
    ref = oracle.run_query(fact, dim, q, extra)
    for flags in (0, T.TP_FLAG_NO_DIRECT_AGG):
        e = T.Engine(page_bytes=2 << 20, n_pages=256, batch_rows=65_536, flags=flags)
        try:
            with _run(e, fact, dim, q, placement=T.TP_HOST_PAGES, extra=extra) as r:
                assert_matches_oracle(r, ref, q["aggs"])
        finally:
            e.close()


def test_fanout_of_duplicated_rows_doubles_the_plain_join():
    fact, dim = _tiny(83, 300_000, 10_000, 12_000)
    twice = {k: np.concatenate([v, v]) for k, v in dim.items()}
    e = T.Engine(page_bytes=8 << 20, n_pages=64, batch_rows=1 << 20)
    try:
        with _run(e, fact, dim, W.q_lowcard()) as one, _run(e, fact, twice, _fanout_query()) as two:
            assert np.array_equal(one.keys(), two.keys())
            assert np.array_equal(2 * one.counts(), two.counts())
    finally:
        e.close()


def test_fanout_refusals():
    fact, dim = _fanout_tables(84, 10_000, 500, 600)
    e = T.Engine(page_bytes=8 << 20, n_pages=16, batch_rows=1 << 20)
    try:
        ft = e.table_from_numpy(fact, placement=T.TP_DEVICE)
        dt = e.table_from_numpy(dim, placement=T.TP_DEVICE)
        with pytest.raises(T.TPError) as err:
            e.plan(ft, dt, _fanout_query(), join_partitions=16)
        assert err.value.status == "invalid"
        p = e.plan(ft, dt, _fanout_query())
        with pytest.raises(T.TPError) as err:
            T.Batch(e, [p])
        assert err.value.status == "invalid"
        with pytest.raises(T.TPError) as err:      # the same keys without fan-out are duplicates
            q = W.q_lowcard()
            p2 = e.plan(ft, dt, q)
            try:
                p2.execute()
            finally:
                p2.destroy()
        assert err.value.status == "dup_key"
        p.destroy()
        ft.destroy()
        dt.destroy()
    finally:
        e.close()


def test_empty_sides_of_fanout_and_star_joins():
    """A further dimension without rows, a fan-out side whose predicate admits
    nothing, lookahead filters over empty key sets, and a split aggregation
    over a fan-out star join: each equals the oracle (mostly: no groups)."""
    fact, dim = _fanout_tables(85, 120_000, 3_000, 3_500)
    _, _, extra = _star_tiny(85, 10, [10, 50], [10, 60])
    fact["fk2"] = datagen.uniform(5085, 7, np.int64, 120_000, 0, 59)
    empty = {k: v[:0] for k, v in extra[0].items()}
    base = _fanout_query()
    base["extra_joins"] = [dict(fact_col="fk2", dim_col="pk")]
    base["group"] = [("fact", "flag", 2), ("dim", "attr", 5), ("dim1", "band", 2)]
    cases = [
        (base, [empty], {}),                                                       # no partner anywhere
        (dict(base, dim_filter=dict(col="attr", lo=40, hi=50)), extra, dict(lip=T.TP_LIP_ON)),
        (dict(base, extra_joins=[dict(fact_col="fk2", dim_col="pk", dim_filter=dict(col="attr", lo=99, hi=99))]),
         extra, dict(lip=T.TP_LIP_ON)),
    ]
    e = T.Engine(page_bytes=8 << 20, n_pages=64, batch_rows=1 << 20)
    try:
        for q, xd, kw in cases:
            ref = oracle.run_query(fact, dim, q, xd)
            assert ref.n_groups == 0
            with _run(e, fact, dim, q, extra=xd, **kw) as r:
                assert_matches_oracle(r, ref, q["aggs"])
    finally:
        e.close()
    # many groups under a budget that forces key-range passes
    fact["okey"] = (np.arange(120_000, dtype=np.int64) * 7919) % 30_011
    q = dict(base, group=[("fact", "okey", 15), ("dim", "attr", 5), ("dim1", "band", 2)])
    ref = oracle.run_query(fact, dim, q, extra)
    for flags in (0, T.TP_FLAG_NO_DIRECT_AGG):
        e = T.Engine(page_bytes=8 << 20, n_pages=64, batch_rows=1 << 20, flags=flags)
        try:
            with _run(e, fact, dim, q, extra=extra) as r:
                assert_matches_oracle(r, ref, q["aggs"])
            peak = e.stats()["peak_reserved"]
        finally:
            e.close()
        e = T.Engine(page_bytes=8 << 20, n_pages=64, batch_rows=1 << 20, flags=flags)
        try:
            e.set_budget(int(peak * 0.8))
            try:
                r = _run(e, fact, dim, q, extra=extra)
            except T.TPError as err:
                assert err.status == "budget"
                continue
            with r:
                assert_matches_oracle(r, ref, q["aggs"])
        finally:
            e.close()
