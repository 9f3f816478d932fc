"""GPU path vs the CPU oracle, element by element, through the C ABI.

Sizes span several tiles and a ragged tail; the full-size star workload
(60M fact rows, 2M-row dimension) is checked against the oracle too."""
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
    e = T.Engine(page_bytes=4 << 20, n_pages=512, batch_rows=1 << 20)
    yield e
    e.close()


def run_gpu(eng, fact, dim, query, placement=T.TP_DEVICE, batch_rows=0, **plan_kw):
    ft = eng.table_from_numpy(fact, placement=placement, batch_rows=batch_rows)
    dt = eng.table_from_numpy(dim, placement=placement, batch_rows=batch_rows) if dim is not None else None
    try:
        p = eng.plan(ft, dt, query, **plan_kw)
        try:
            return p.execute()
        finally:
            p.destroy()
    finally:
        ft.destroy()
        if dt is not None:
            dt.destroy()


def check(eng, fact, dim, query, **kw):
    ref = oracle.run_query(fact, dim, query)
    with run_gpu(eng, fact, dim, query, **kw) as res:
        assert_matches_oracle(res, ref, query["aggs"])
    return ref


def test_config1_full_size(eng):
    wl = W.config1()
    ref = check(eng, wl.fact, wl.dim, wl.query)
    assert ref.n_groups == 150


@pytest.mark.parametrize("n_fact,n_dim", [(1, 1), (127, 10), (128, 100), (129, 100), (1000, 1),
                                          (65_537, 10_000), (300_001, 777)])
def test_config1_ragged(eng, n_fact, n_dim):
    wl = W.config1(n_fact=n_fact, n_dim=n_dim)
    check(eng, wl.fact, wl.dim, wl.query)


@pytest.mark.parametrize("which,strategy", [("a", T.TP_AGG_AUTO), ("a", T.TP_AGG_GLOBAL),
                                            ("b", T.TP_AGG_AUTO), ("b2", T.TP_AGG_AUTO)])
@pytest.mark.parametrize("sparse", [False, True])
def test_config2_small(eng, which, strategy, sparse):
    """sparse: unique sparse int64 dimension keys, so the join is hashed."""
    wl = W.config2(which, n_fact=3_000_017, n_dim=300_000, sparse_keys=sparse)
    check(eng, wl.fact, wl.dim, wl.query, agg_strategy=strategy)


def test_torch_wrapped_columns(eng):
    import torch
    wl = W.config1(n_fact=500_003)
    ref = oracle.run(wl)
    ft = eng.table_from_torch({k: torch.from_numpy(v).cuda() for k, v in wl.fact.items()})
    dt = eng.table_from_torch({k: torch.from_numpy(v).cuda() for k, v in wl.dim.items()})
    p = eng.plan(ft, dt, wl.query)
    for _ in range(2):   # second run reuses the plan's sampled selectivity
        with p.execute() as res:
            assert_matches_oracle(res, ref, wl.query["aggs"])
    p.destroy()
    ft.destroy()
    dt.destroy()


@pytest.mark.parametrize("batch_rows", [65_536, 99_991, 1_000_000])
def test_paged_streaming(eng, batch_rows):
    wl = W.config1(n_fact=2_000_003, n_dim=10_000)
    check(eng, wl.fact, wl.dim, wl.query, placement=T.TP_HOST_PAGES, batch_rows=batch_rows)


@pytest.mark.parametrize("depth", [0, 1, 4])
def test_prefetch_depths_agree(depth):
    wl = W.config1(n_fact=700_001, n_dim=5_000)
    ref = oracle.run(wl)
    e = T.Engine(page_bytes=1 << 20, n_pages=256, batch_rows=50_000, prefetch_depth=depth)
    try:
        with run_gpu(e, wl.fact, wl.dim, wl.query, placement=T.TP_HOST_PAGES) as res:
            assert_matches_oracle(res, ref, wl.query["aggs"])
        st = e.stats()
        assert st["batches"] == 15 and st["h2d_bytes"] > 0
    finally:
        e.close()


@pytest.mark.parametrize("depth,pinned", [(0, False), (3, False), (2, True), (0, True)])
def test_copy_options_agree(depth, pinned):
    """Prefetch depth and the per-batch pinned buffers (the no-pool ablation)
    set after the engine starts change nothing in the result."""
    wl = W.config1(n_fact=700_001, n_dim=5_000)
    ref = oracle.run(wl)
    e = T.Engine(page_bytes=1 << 20, n_pages=256, batch_rows=50_000)
    try:
        e.set_copy_options(depth, pinned)
        with run_gpu(e, wl.fact, wl.dim, wl.query, placement=T.TP_HOST_PAGES) as res:
            assert_matches_oracle(res, ref, wl.query["aggs"])
        with pytest.raises(T.TPError):
            e.set_copy_options(-1)
    finally:
        e.close()


def test_int64_keys_and_sparse_pk(eng):
    dim = W.config3_dim(n_dim=100_000)
    fact = W.config3_fact(0, 1_000_003, n_dim=100_000)
    q = W.q_lowcard()
    check(eng, fact, dim, q)
    check(eng, fact, dim, q, placement=T.TP_HOST_PAGES, batch_rows=300_000)


@pytest.mark.parametrize("seed,n_fact,n_dim,span,cutoff", [
    (0, 2000, 200, 250, W.CUTOFF_98), (1, 1500, 150, 150, W.N_DAYS - 1), (2, 1000, 100, 400, 1000),
    (3, 777, 1, 2, 2000), (4, 500, 120, 120, -1), (5, 0, 50, 50, W.CUTOFF_98), (6, 300, 0, 10, W.CUTOFF_98)])
def test_tiny_cases(eng, seed, n_fact, n_dim, span, cutoff):
    fact, dim = _tiny(seed, n_fact, n_dim, span)
    q = W.q_lowcard(cutoff)
    check(eng, fact, dim, q)
    check(eng, fact, dim, q, agg_strategy=T.TP_AGG_GLOBAL)


def test_other_query_shapes(eng):
    fact, dim = _tiny(8, 50_000, 600, 800, signed=True)
    queries = [
        dict(filter=None, join=dict(fact_col="fk", dim_col="pk"), group=[("dim", "attr", 5)],
             aggs=[("sum", "price"), ("avg", "qty"), ("sum_mul_sub", "qty", -7, "price")]),
        dict(filter=dict(col="date", lo=300, hi=2000), join=None,
             group=[("fact", "flag", 2), ("fact", "status", 1)],
             aggs=[("sum_mul_sub", "price", 100, "disc"), ("count",), ("avg", "price")]),
        dict(filter=None, join=None, group=[], aggs=[("sum", "qty"), ("count",)]),
        dict(filter=None, join=dict(fact_col="fk", dim_col="pk"), group=[("fact", "qty", 64)],
             aggs=[("count",)]),
        dict(filter=dict(col="qty", lo=-100, hi=2500), join=dict(fact_col="fk", dim_col="pk"),
             group=[("dim", "attr", 5), ("fact", "flag", 2)], aggs=[("count",), ("avg", "disc")]),
    ]
    for q in queries:
        check(eng, fact, dim, q)
        check(eng, fact, dim, q, agg_strategy=T.TP_AGG_GLOBAL)


def test_sentinel_keys(eng):
    """Keys equal to the all-ones empty-slot pattern: join key -1 (32- and
    64-bit tables) and a packed group key of 2^64-1."""
    n = 10_000
    for kt in (np.int32, np.int64):
        dim = dict(pk=np.array([-1, 0, 5, 7], kt), attr=np.array([3, 1, 2, 4], np.int32))
        fk = datagen.uniform(3, 1, np.int64, n, -2, 8).astype(kt)
        fact = dict(fk=fk, qty=datagen.uniform(3, 2, np.int64, n, -1000, 1000),
                    g=datagen.uniform(3, 3, np.int64, n, -2, 1))
        q = dict(filter=None, join=dict(fact_col="fk", dim_col="pk"),
                 group=[("fact", "g", 64)], aggs=[("sum", "qty"), ("count",)])
        check(eng, fact, dim, q)
        q2 = dict(q, group=[("dim", "attr", 3)])
        check(eng, fact, dim, q2)


def test_errors(eng):
    fact, dim = _tiny(9, 5_000, 200, 200)
    bad = dict(dim)
    bad["pk"] = dim["pk"].copy()
    bad["pk"][5] = bad["pk"][6]
    with pytest.raises(T.TPError) as e:
        run_gpu(eng, fact, bad, W.q_lowcard())
    assert e.value.status == "dup_key"
    with pytest.raises(T.TPError) as e:
        run_gpu(eng, fact, dim, W.q_lowcard(cutoff=W.N_DAYS - 1, attr_bits=4))
    assert e.value.status == "range"
    # an out-of-range attribute on a dimension row no fact row reaches is fine
    dim2 = {k: v.copy() for k, v in dim.items()}
    fact2 = {k: v.copy() for k, v in fact.items()}
    fact2["fk"][fact2["fk"] == dim2["pk"][0]] = dim2["pk"][1]
    dim2["attr"][0] = 99
    check(eng, fact2, dim2, W.q_lowcard())


def test_repeat_is_deterministic(eng):
    wl = W.config2("b2", n_fact=1_000_000, n_dim=100_000)
    ft = eng.table_from_numpy(wl.fact, placement=T.TP_DEVICE)
    dt = eng.table_from_numpy(wl.dim, placement=T.TP_DEVICE)
    p = eng.plan(ft, dt, wl.query)
    outs = []
    for _ in range(3):
        with p.execute() as r:
            outs.append((r.keys(), r.counts(), r.sum_words(0)))
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            assert np.array_equal(x, y)
    p.destroy()
    ft.destroy()
    dt.destroy()


def test_budget_refusal_and_release(eng):
    wl = W.config1(n_fact=100_000)
    used0, cap0 = eng.budget()
    eng.set_budget(used0 + 1000)
    try:
        with pytest.raises(T.TPError) as e:
            run_gpu(eng, wl.fact, wl.dim, wl.query, placement=T.TP_HOST_PAGES)
        assert e.value.status == "budget"
    finally:
        eng.set_budget(cap0)
    assert eng.budget()[0] == used0
    check(eng, wl.fact, wl.dim, wl.query)
    assert eng.budget()[0] == used0


@pytest.mark.parametrize("flags", [0, T.TP_FLAG_EXACT_ONLY, T.TP_FLAG_NO_STAGED, T.TP_FLAG_NO_DIRECT_JOIN,
                                   T.TP_FLAG_NO_STAGED | T.TP_FLAG_NO_DIRECT_JOIN, T.TP_FLAG_NO_JIT,
                                   T.TP_FLAG_NO_JIT | T.TP_FLAG_EXACT_ONLY, T.TP_FLAG_NO_JIT | T.TP_FLAG_NO_DIRECT_JOIN,
                                   T.TP_FLAG_NO_DIRECT_AGG, T.TP_FLAG_RAW_PAGES])
def test_every_kernel_path(flags):
    """Staged 64-bit (bounds prove no overflow), staged exact 128-bit, the
    plain-load kernel, hashed instead of direct-mapped join tables, and the
    run-time compiled and ahead-of-time staged kernels all give the oracle's
    result."""
    e = T.Engine(page_bytes=4 << 20, n_pages=256, batch_rows=700_000, flags=flags)
    try:
        wl = W.config2("a", n_fact=2_000_011, n_dim=200_000)
        for placement in (T.TP_DEVICE, T.TP_HOST_PAGES):
            check(e, wl.fact, wl.dim, wl.query, placement=placement)
        fact, dim = _tiny(8, 40_000, 600, 800, signed=True)
        q = dict(filter=dict(col="qty", lo=-100, hi=2500), join=dict(fact_col="fk", dim_col="pk"),
                 group=[("dim", "attr", 5), ("fact", "flag", 2)],
                 aggs=[("count",), ("avg", "disc"), ("sum_mul_sub", "price", -3, "qty"), ("sum", "price")])
        check(e, fact, dim, q)
        # values whose sums need all 128 bits: the exact path must carry
        n = 5_000
        big = dict(a=np.full(n, (1 << 62) + 12345, np.int64), b=np.full(n, -(1 << 62), np.int64),
                   g=(np.arange(n) % 3).astype(np.uint8), d=datagen.uniform(4, 4, np.int32, n, 0, 9))
        qb = dict(filter=dict(col="d", lo=1, hi=8), join=None, group=[("fact", "g", 2)],
                  aggs=[("sum_mul_sub", "a", (1 << 62), "b"), ("sum", "a"), ("avg", "b")])
        check(e, big, None, qb)
    finally:
        e.close()


JIT_QUERIES = {
    # int64 filter column, a uint8 field wider than 8 bits, a product in the
    # 64-bit carry mode
    "i64-filter-wide-u8": dict(filter=dict(col="price", lo=200_000, hi=9_000_000),
                               join=dict(fact_col="fk", dim_col="pk"),
                               group=[("fact", "flag", 8), ("fact", "status", 1)],
                               aggs=[("sum_mul_sub", "price", 100, "disc"), ("count",)]),
    "no-filter-no-join": dict(filter=None, join=None, group=[("fact", "status", 1), ("fact", "flag", 2)],
                              aggs=[("sum", "qty"), ("avg", "disc")]),
    "count-only": dict(filter=dict(col="date", lo=0, hi=1800), join=dict(fact_col="fk", dim_col="pk"),
                       group=[("dim", "attr", 5)], aggs=[("count",)]),
}


@pytest.mark.parametrize("name", sorted(JIT_QUERIES))
@pytest.mark.parametrize("flags", [0, T.TP_FLAG_NO_DIRECT_JOIN])
def test_jit_shapes_match_oracle(name, flags):
    """Plan shapes compiled at run time give the oracle's result, and the
    run-time compiled kernel is the one that ran."""
    wl = W.config2("a", n_fact=1_500_007, n_dim=100_000)
    e = T.Engine(page_bytes=4 << 20, n_pages=256, flags=flags)
    try:
        s0 = e.stats()
        check(e, wl.fact, wl.dim, JIT_QUERIES[name])
        s1 = e.stats()
        assert s1["jit_failures"] == 0
        assert s1["jit_launches"] > s0["jit_launches"]
    finally:
        e.close()


def test_jit_fact_field_range_error():
    """A fact-side group field outside its bit width is reported by the
    run-time compiled kernel too."""
    wl = W.config2("a", n_fact=300_007, n_dim=100_000)
    e = T.Engine(page_bytes=4 << 20, n_pages=64)
    try:
        q = dict(filter=None, join=None, group=[("fact", "qty", 3)], aggs=[("count",)])
        with pytest.raises(T.TPError) as err:
            run_gpu(e, wl.fact, wl.dim, q)
        assert err.value.status == "range"
        assert e.stats()["jit_launches"] > 0
    finally:
        e.close()


@pytest.mark.parametrize("flags", [0, T.TP_FLAG_NO_DIRECT_AGG, T.TP_FLAG_EXACT_ONLY,
                                   T.TP_FLAG_EXACT_ONLY | T.TP_FLAG_NO_DIRECT_AGG, T.TP_FLAG_NO_STAGED])
@pytest.mark.parametrize("which", ["b", "b2"])
def test_many_groups_direct_and_hashed(flags, which):
    """Many groups: the direct-addressed table (dense order keys, sorted output
    without a sort) and the hashed table (with compaction and radix sort) give
    the oracle's result, in 64-bit and exact accumulation."""
    wl = W.config2(which, n_fact=2_400_011, n_dim=150_000)
    e = T.Engine(page_bytes=8 << 20, n_pages=256, batch_rows=1_000_000, flags=flags)
    try:
        check(e, wl.fact, wl.dim, wl.query)
        check(e, wl.fact, wl.dim, wl.query, placement=T.TP_HOST_PAGES)
    finally:
        e.close()


@pytest.mark.parametrize("flags", [0, T.TP_FLAG_RAW_PAGES])
def test_narrow_pages_round_trip(flags):
    """Host-page columns stored narrow (per batch: value - minimum in 1, 2 or 4
    bytes) or at full width give the oracle's result, for negative values,
    spans that need every width, and spans too wide to narrow."""
    n = 300_017
    rng = np.random.default_rng(11)
    fact = dict(
        fk=rng.integers(-50, 50, n).astype(np.int64),                       # negative, 1 byte
        w2=rng.integers(-30_000, 30_000, n).astype(np.int64),               # 2 bytes
        w4=rng.integers(-(1 << 31), 1 << 31, n).astype(np.int64),           # 4 bytes
        w8=(rng.integers(0, 1 << 62, n) - (1 << 61)).astype(np.int64),      # full width
        i32=rng.integers(-(1 << 31), (1 << 31) - 1, n).astype(np.int32),    # full width
        d=rng.integers(0, 2557, n).astype(np.int32),
        g=rng.integers(0, 3, n).astype(np.uint8),
    )
    dim = dict(pk=np.arange(-50, 50, dtype=np.int64), attr=(np.arange(100) % 7).astype(np.int32))
    q = dict(filter=dict(col="d", lo=10, hi=2400), join=dict(fact_col="fk", dim_col="pk"),
             group=[("dim", "attr", 3), ("fact", "g", 2)],
             aggs=[("sum", "w2"), ("sum", "w4"), ("sum", "w8"), ("sum", "i32"), ("count",), ("avg", "w2")])
    e = T.Engine(page_bytes=1 << 20, n_pages=256, batch_rows=40_000, flags=flags)
    try:
        check(e, fact, dim, q, placement=T.TP_HOST_PAGES)
        ft = e.table_from_numpy(fact, placement=T.TP_DEVICE)      # placed from (narrow) pages
        dt = e.table_from_numpy(dim, placement=T.TP_DEVICE)
        p = e.plan(ft, dt, q)
        with p.execute() as r:
            assert_matches_oracle(r, oracle.run_query(fact, dim, q), q["aggs"])
        p.destroy(); ft.destroy(); dt.destroy()
    finally:
        e.close()


@pytest.mark.parametrize("chunk", [3_001, 25_001])
@pytest.mark.parametrize("prefetch", [0, 2])
def test_bit_packed_pages_every_width(chunk, prefetch):
    """Host-page columns bit-packed per batch at every width from 1 to 31 bits
    (int64, int32 and uint8 columns; 8 and 16 bits stay byte widths) give the
    oracle's result.  The table is appended in chunks: 3,001-row chunks make
    one batch each, so several of them share a staging slot at row offsets that
    leave a packed stream unaligned to its words; 25,001-row chunks make odd
    batches of 9,999 rows with ragged last ones.  The filter, the join key and a
    group key are packed columns too."""
    n = 60_013
    rng = np.random.default_rng(23)
    fact = dict(
        d=rng.integers(0, 2557, n).astype(np.int32),                 # 12 bits
        fk=rng.integers(-40, 60, n).astype(np.int64),                 # 7 bits, negative
        g=rng.integers(0, 3, n).astype(np.uint8),                     # 2 bits
    )
    names = []
    for bits in range(1, 32):
        lo = int(rng.integers(-(1 << 40), 1 << 40))
        fact[f"q{bits}"] = rng.integers(0, 1 << bits, n).astype(np.int64) + lo
        names.append(f"q{bits}")
        if bits < 31:
            lo32 = int(rng.integers(-(1 << 30), (1 << 30) - (1 << bits)))
            fact[f"i{bits}"] = (rng.integers(0, 1 << bits, n) + lo32).astype(np.int32)
            names.append(f"i{bits}")
        if bits < 8:
            fact[f"u{bits}"] = rng.integers(0, 1 << bits, n).astype(np.uint8)
            names.append(f"u{bits}")
    dim = dict(pk=np.arange(-40, 60, dtype=np.int64), attr=(np.arange(100) % 5).astype(np.int32))
    e = T.Engine(page_bytes=1 << 20, n_pages=512, batch_rows=9_999, prefetch_depth=prefetch)
    try:
        dt = e.table_from_numpy(dim, placement=T.TP_HOST_PAGES)
        for t0 in range(0, len(names), 28):   # a table holds at most 32 columns
            part = {k: fact[k] for k in ("d", "fk", "g")}
            part.update({k: fact[k] for k in names[t0:t0 + 28]})
            ft = e.table_from_chunks({k: v[r:r + chunk] for k, v in part.items()} for r in range(0, n, chunk))
            for k in range(t0, min(t0 + 28, len(names)), 6):   # six sums, a count and an average
                cols = names[k:min(k + 6, t0 + 28)]
                q = dict(filter=dict(col="d", lo=10, hi=2400), join=dict(fact_col="fk", dim_col="pk"),
                         group=[("dim", "attr", 3), ("fact", "g", 2)],
                         aggs=[("sum", c) for c in cols] + [("count",), ("avg", cols[0])])
                p = e.plan(ft, dt, q)
                with p.execute() as r:
                    assert_matches_oracle(r, oracle.run_query(part, dim, q), q["aggs"])
                p.destroy()
            ft.destroy()
        dt.destroy()
    finally:
        e.close()
