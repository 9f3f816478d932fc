"""Sums at the edges of their word sizes, through tp_execute on every kernel
path, against the oracle bit for bit.

Section 4 holds decimals as 128-bit integers, so a sum may leave int64: terms
near 2^62 (and products of two such factors) push the high words of every
accumulator -- shared 128-bit tables, the global table, the fold into the
dense table -- and their AVG takes the wide int128 -> double conversion.

The 32-bit per-CTA tables are chosen by bounding the rows one CTA can see;
the run-time compiled kernel also hands the rows after the last whole tile to
CTA (tiles % grid), which is CTA 0 when the tiles divide evenly.  The boundary
cases below put that CTA's sum exactly one tail past the bound a whole-tile
count would give."""
import numpy as np
import pytest

import oracle
from paper_2508_05029_gb300 import theseus as T
from tests.helpers import assert_matches_oracle

pytestmark = pytest.mark.gpu

JIT_TILE = 24 * 32 * 2    # rows per tile of the run-time compiled dense kernel


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_05029_gb300 import build
    build.build()


def _num_sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def _run(fact, dim, q, flags=0, placement=T.TP_DEVICE, batch_rows=0, **plan_kw):
    e = T.Engine(page_bytes=4 << 20, n_pages=64, batch_rows=1 << 22, flags=flags)
    try:
        tabs = [e.table_from_numpy(fact, placement=placement, batch_rows=batch_rows)]
        if dim is not None:
            tabs.append(e.table_from_numpy(dim, placement=placement, batch_rows=batch_rows))
        p = e.plan(tabs[0], tabs[1] if dim is not None else None, q, **plan_kw)
        try:
            ref = oracle.run_query(fact, dim, q)
            with p.execute() as r:
                assert_matches_oracle(r, ref, q["aggs"])
            return ref, e.stats()
        finally:
            p.destroy()
            for t in tabs:
                t.destroy()
    finally:
        e.close()


# ------------------------------------------------- the 32-bit bound and the tail

def _tail_case(n, v, lo=0, flag_bits=0):
    """Column x: lo in row 0, lo + v elsewhere, so its span is exactly v."""
    x = np.full(n, lo + v, np.int64)
    x[0] = lo
    fact = dict(x=x, f=(np.arange(n) % 3).astype(np.uint8))
    group = [("fact", "f", 2)] if flag_bits else []
    q = dict(filter=None, join=None, group=group, aggs=[("sum", "x"), ("avg", "x"), ("count",)])
    return fact, q


@pytest.mark.parametrize("tiles_per_cta,extra_tiles,tail", [(1, 0, JIT_TILE - 1), (2, 0, JIT_TILE - 1),
                                                            (1, 0, 1), (1, 5, JIT_TILE - 1), (3, 0, 777)])
@pytest.mark.parametrize("grouped", [False, True])
def test_low_word_bound_counts_the_tail(tiles_per_cta, extra_tiles, tail, grouped):
    """v = floor((2^32 - 1) / whole-tile rows per CTA): a bound that ignored the
    tail would pick 32-bit low words, and the tail CTA would wrap them."""
    sms = _num_sms()
    tiles = tiles_per_cta * sms + extra_tiles
    n = tiles * JIT_TILE + tail
    share = -(-tiles // sms) * JIT_TILE
    v = 0xFFFFFFFF // share
    fact, q = _tail_case(n, v, flag_bits=grouped)
    _, st = _run(fact, None, q)
    assert st["jit_launches"] >= 1   # the run-time compiled kernel took the rows


@pytest.mark.parametrize("v,lo", [(1 << 40, 0), (1 << 40, -(1 << 39)), ((1 << 45) + 12345, 7),
                                  (0xFFFFFFFF // (2 * JIT_TILE - 1) + 1, 0)])
def test_carry_words_with_tail(v, lo):
    """Spans past 32 bits keep a carry word per group; sums stay in int64."""
    n = _num_sms() * JIT_TILE + JIT_TILE - 1
    fact, q = _tail_case(n, v, lo=lo, flag_bits=2)
    _, st = _run(fact, None, q)
    assert st["jit_launches"] >= 1


def test_tail_bound_with_join_and_product():
    """The same boundary through a direct join and SUM(a * (K - b))."""
    sms = _num_sms()
    n = sms * JIT_TILE + JIT_TILE - 1
    k, b = 100, 99                                  # K - b = 1: each term equals a
    a = np.full(n, 0xFFFFFFFF // JIT_TILE, np.int64)
    a[0] = 0
    fact = dict(fk=(np.arange(n) % 1000).astype(np.int32), a=a, b=np.full(n, b, np.int64))
    dim = dict(pk=np.arange(1000, dtype=np.int32), attr=(np.arange(1000) % 3).astype(np.int32))
    q = dict(filter=None, join=dict(fact_col="fk", dim_col="pk"), group=[("dim", "attr", 2)],
             aggs=[("sum_mul_sub", "a", k, "b"), ("count",)])
    _, st = _run(fact, dim, q)
    assert st["jit_launches"] >= 1


# ------------------------------------------------------- sums beyond int64

PATHS = [("jit", 0), ("aot_staged", T.TP_FLAG_NO_JIT), ("plain", T.TP_FLAG_NO_STAGED),
         ("exact_only", T.TP_FLAG_EXACT_ONLY), ("hashed_join", T.TP_FLAG_NO_DIRECT_JOIN)]


def _wide(seed, n, n_dim=5000, n_okeys=40_000):
    """Fact terms near 2^62 (mostly positive, so group sums pass 2^64 and AVG
    takes the wide conversion) and products of two 2^40-scale factors."""
    rng = np.random.default_rng(0x51DE + seed)
    big = rng.integers(1 << 61, 1 << 62, n, dtype=np.int64)
    big[rng.random(n) < 0.1] *= -1
    fact = dict(
        fk=rng.integers(-5, n_dim + 5, n).astype(np.int32),
        d=rng.integers(0, 100, n).astype(np.int32),
        big=big,
        f40=rng.integers(-(1 << 40), 1 << 40, n, dtype=np.int64),
        g40=rng.integers(-(1 << 40), 1 << 40, n, dtype=np.int64),
        flag=rng.integers(0, 3, n).astype(np.uint8),
        ok=rng.permutation(np.repeat(np.arange(n_okeys, dtype=np.int64) * 7 + 3, -(-n // n_okeys))[:n]),
    )
    dim = dict(pk=rng.permutation(n_dim).astype(np.int32), attr=rng.integers(0, 25, n_dim).astype(np.int32))
    return fact, dim


def _wide_queries():
    aggs = [("sum", "big"), ("avg", "big"), ("sum_mul_sub", "f40", 1 << 20, "g40"), ("count",)]
    join = dict(fact_col="fk", dim_col="pk")
    return {
        "lowcard": dict(filter=dict(col="d", lo=0, hi=97), join=join,
                        group=[("fact", "flag", 2), ("dim", "attr", 5)], aggs=aggs),
        "ungrouped": dict(filter=None, join=join, group=[], aggs=aggs),
        "manygroups": dict(filter=dict(col="d", lo=0, hi=97), join=join, group=[("fact", "ok", 64)], aggs=aggs),
    }


@pytest.mark.parametrize("path,flags", PATHS)
@pytest.mark.parametrize("which", ["lowcard", "ungrouped", "manygroups"])
@pytest.mark.parametrize("placement", [T.TP_DEVICE, T.TP_HOST_PAGES])
def test_sums_beyond_int64(path, flags, which, placement):
    fact, dim = _wide([p for p, _ in PATHS].index(path) * 3 + ["lowcard", "ungrouped", "manygroups"].index(which),
                      300_007)
    q = _wide_queries()[which]
    ref, _ = _run(fact, dim, q, flags=flags, placement=placement, batch_rows=100_000)
    # the high words really carry, and AVG takes the wide conversion
    hi = ref.sums[:, 0, 1].view(np.int64)
    assert np.any((hi != 0) & (hi != -1))
    assert np.any(ref.sums[:, 2, 1].view(np.int64) != (ref.sums[:, 2, 0].view(np.int64) >> 63))


@pytest.mark.parametrize("strategy,flags", [(T.TP_AGG_GLOBAL, 0), (T.TP_AGG_GLOBAL, T.TP_FLAG_NO_DIRECT_AGG),
                                            (T.TP_AGG_GLOBAL, T.TP_FLAG_NO_STAGED),
                                            (T.TP_AGG_GLOBAL, T.TP_FLAG_EXACT_ONLY)])
def test_sums_beyond_int64_global_table(strategy, flags):
    """Few groups forced through the global table (direct and hashed)."""
    fact, dim = _wide(77, 200_003)
    q = _wide_queries()["lowcard"]
    _run(fact, dim, q, flags=flags, agg_strategy=strategy)
    _run(fact, dim, q, flags=flags, agg_strategy=strategy, placement=T.TP_HOST_PAGES, batch_rows=65_536)


def test_extreme_terms_wrap_like_the_oracle():
    """INT64_MIN/MAX terms and products at the int128 limits."""
    n = 50_021
    rng = np.random.default_rng(99)
    pick = rng.integers(0, 4, n)
    a = np.where(pick == 0, np.iinfo(np.int64).min, np.where(pick == 1, np.iinfo(np.int64).max,
                                                             rng.integers(-(1 << 63), (1 << 63) - 1, n,
                                                                          dtype=np.int64)))
    b = np.where(rng.random(n) < 0.5, np.iinfo(np.int64).min, np.iinfo(np.int64).max).astype(np.int64)
    fact = dict(a=a.astype(np.int64), b=b, flag=rng.integers(0, 3, n).astype(np.uint8))
    q = dict(filter=None, join=None, group=[("fact", "flag", 2)],
             aggs=[("sum", "a"), ("avg", "a"), ("sum_mul_sub", "a", -1, "b"), ("count",)])
    for flags in (0, T.TP_FLAG_NO_JIT, T.TP_FLAG_NO_STAGED):
        _run(fact, None, q, flags=flags)
        _run(fact, None, q, flags=flags, agg_strategy=T.TP_AGG_GLOBAL)
