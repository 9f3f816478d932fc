"""Pins for the CPU oracle against things other than itself.

* brute force: nested-loop join + linear group scan in Python integers on tiny
  inputs (misses, empty results, all-pass and none-pass filters, signed values);
* closed form: a modular dataset whose per-group counts and sums are
  arithmetic-series formulas;
* invariants: group counts sum to the joined row count, grouped sums add up to
  the ungrouped sum, row-order independence;
* a second, independent int64 evaluation with PyTorch CPU tensor ops;
* the int128 -> double conversion against Python's correctly rounded int->float.
"""
import math

import numpy as np
import pytest

import datagen
import oracle
from datagen import workloads as W
from tests import bruteforce

I64_MIN, I64_MAX = W.I64_MIN, W.I64_MAX


def _check_against_brute(fact, dim, query):
    ref = bruteforce.evaluate(fact, dim, query)
    got = oracle.run_query(fact, dim, query)
    assert got.n_groups == len(ref)
    for g, (key, count, sums, avgs) in enumerate(ref):
        assert int(got.keys[g]) == key
        assert int(got.counts[g]) == count
        for a, ag in enumerate(query["aggs"]):
            assert got.sum_int(g, a) == sums[a], (g, a, ag)
            if ag[0] == "avg":
                assert got.avgs[g, a] == avgs[a]
    return got


def _tiny(seed, n_fact, n_dim, key_span, signed=False):
    """Tiny star tables; fk drawn from a span wider than the dimension keys so
    that some rows miss the join."""
    s = 1000 + seed
    dim = dict(
        pk=datagen.fill(s, 1, datagen.PERM, np.int32, n_dim, b=max(n_dim, 1)) if n_dim else
        np.zeros(0, np.int32),
        attr=datagen.uniform(s, 2, np.int32, n_dim, 0, 24),
    )
    lo_m = -5000 if signed else 100
    fact = dict(
        fk=datagen.uniform(s, 3, np.int32, n_fact, 0, key_span - 1),
        date=datagen.uniform(s, 4, np.int32, n_fact, 0, W.N_DAYS - 1),
        qty=datagen.uniform(s, 5, np.int64, n_fact, lo_m, 5000),
        price=datagen.uniform(s, 6, np.int64, n_fact, -10_500_000 if signed else 90_000, 10_500_000),
        disc=datagen.uniform(s, 7, np.int64, n_fact, 0, 10),
        flag=datagen.uniform(s, 8, np.uint8, n_fact, 0, 2),
        status=datagen.uniform(s, 9, np.uint8, n_fact, 0, 1),
    )
    return fact, dim


@pytest.mark.parametrize("seed,n_fact,n_dim,span,cutoff", [
    (0, 2000, 200, 250, W.CUTOFF_98),    # ~20% misses
    (1, 1500, 150, 150, W.N_DAYS - 1),   # all rows pass the filter and match
    (2, 1000, 100, 400, 1000),           # selective filter, many misses
    (3, 777, 1, 2, 2000),                # single-row dimension
    (4, 500, 120, 120, -1),              # no row passes the filter
    (5, 0, 50, 50, W.CUTOFF_98),         # empty fact table
    (6, 300, 0, 10, W.CUTOFF_98),        # empty dimension: nothing joins
])
def test_lowcard_matches_bruteforce(seed, n_fact, n_dim, span, cutoff):
    fact, dim = _tiny(seed, n_fact, n_dim, span)
    q = W.q_lowcard(cutoff)
    got = _check_against_brute(fact, dim, q)
    if cutoff < 0 or n_fact == 0 or n_dim == 0:
        assert got.n_groups == 0


def test_filter_bounds_are_inclusive():
    fact, dim = _tiny(7, 1200, 100, 100)
    for lo, hi in [(500, 500), (0, 0), (W.N_DAYS - 1, W.N_DAYS - 1), (100, 125)]:
        q = W.q_lowcard()
        q["filter"] = dict(col="date", lo=lo, hi=hi)
        got = _check_against_brute(fact, dim, q)
        want = int(((fact["date"] >= lo) & (fact["date"] <= hi) & (fact["fk"] < 100)).sum())
        assert int(got.counts.sum()) == want


def test_signed_values_and_other_shapes():
    fact, dim = _tiny(8, 1500, 60, 80, signed=True)
    # dimension-only key, fact-only key, no join, no filter
    queries = [
        dict(filter=None, join=dict(fact_col="fk", dim_col="pk"), group=[("dim", "attr", 5)],
             aggs=[("sum", "price"), ("avg", "qty"), ("sum_mul_sub", "qty", -7, "price")]),
        dict(filter=dict(col="date", lo=300, hi=2000), join=None,
             group=[("fact", "flag", 2), ("fact", "status", 1)],
             aggs=[("sum_mul_sub", "price", 100, "disc"), ("count",), ("avg", "price")]),
        dict(filter=None, join=None, group=[], aggs=[("sum", "qty"), ("count",)]),
        dict(filter=None, join=dict(fact_col="fk", dim_col="pk"),
             group=[("fact", "qty", 64)], aggs=[("count",)]),
    ]
    for q in queries:
        _check_against_brute(fact, dim, q)


def test_errors_duplicate_key_and_range():
    fact, dim = _tiny(9, 100, 20, 20)
    dim["pk"][5] = dim["pk"][6]
    with pytest.raises(oracle.OracleError) as e:
        oracle.run_query(fact, dim, W.q_lowcard())
    assert e.value.status == "dup_key"
    with pytest.raises(ValueError, match="dup_key"):
        bruteforce.evaluate(fact, dim, W.q_lowcard())
    fact, dim = _tiny(9, 100, 20, 20)
    q = W.q_lowcard(cutoff=W.N_DAYS - 1, attr_bits=4)   # attr up to 24 needs 5 bits
    with pytest.raises(oracle.OracleError) as e:
        oracle.run_query(fact, dim, q)
    assert e.value.status == "range"
    bad = dict(W.q_lowcard())
    bad["group"] = [("fact", "flag", 40), ("fact", "status", 30)]  # 70 bits
    with pytest.raises(oracle.OracleError) as e:
        oracle.run_query(fact, dim, bad)
    assert e.value.status == "invalid"


@pytest.mark.parametrize("seed,lo,hi", [
    (20, 3, 10),            # a band of attribute values
    (21, 7, 7),             # a single value: inclusive bounds
    (22, 0, 24),            # every dimension row passes: same as no predicate
    (23, 30, 40),           # none passes: empty result
    (24, -5, 2),            # the low edge
])
def test_dim_filter_matches_bruteforce(seed, lo, hi):
    fact, dim = _tiny(seed, 1500, 180, 220)
    q = dict(W.q_lowcard(), dim_filter=dict(col="attr", lo=lo, hi=hi))
    got = _check_against_brute(fact, dim, q)
    live = set(int(k) for k, a in zip(dim["pk"], dim["attr"]) if lo <= a <= hi)
    want = sum(1 for fk, dt in zip(fact["fk"], fact["date"]) if int(fk) in live and dt <= W.CUTOFF_98)
    assert int(got.counts.sum()) == want
    if lo <= 0 and hi >= 24:   # all rows admitted: the query without the predicate
        plain = oracle.run_query(fact, dim, W.q_lowcard())
        assert np.array_equal(plain.keys, got.keys) and np.array_equal(plain.sums, got.sums)
    if lo > 24:
        assert got.n_groups == 0


def test_dim_filter_duplicates_only_among_admitted_rows():
    fact, dim = _tiny(25, 400, 40, 40)
    dim["pk"][5] = dim["pk"][6]
    dim["attr"][5], dim["attr"][6] = 1, 20
    q = dict(W.q_lowcard(), dim_filter=dict(col="attr", lo=10, hi=24))   # row 5 is out: no clash
    _check_against_brute(fact, dim, q)
    q = dict(W.q_lowcard(), dim_filter=dict(col="attr", lo=0, hi=24))    # both in: duplicate key
    with pytest.raises(oracle.OracleError) as e:
        oracle.run_query(fact, dim, q)
    assert e.value.status == "dup_key"
    with pytest.raises(ValueError, match="dup_key"):
        bruteforce.evaluate(fact, dim, q)


def _star_tiny(seed, n_fact, sizes, spans):
    """A fact table with one foreign key per dimension (fk, fk2, fk3, drawn from
    spans wider than the keys, so some rows miss) and dimensions of the given
    sizes with permuted unique keys and a 0..24 attribute."""
    fact, dim = _tiny(seed, n_fact, sizes[0], spans[0])
    s = 2000 + seed
    extra = []
    for j, (n, span) in enumerate(zip(sizes[1:], spans[1:])):
        extra.append(dict(
            pk=datagen.fill(s, 10 + j, datagen.PERM, np.int64, n, b=max(n, 1)) if n else np.zeros(0, np.int64),
            attr=datagen.uniform(s, 20 + j, np.int32, n, 0, 24),
            band=datagen.uniform(s, 30 + j, np.uint8, n, 0, 3)))
        fact[f"fk{j + 2}"] = datagen.uniform(s, 40 + j, np.int64, n_fact, 0, span - 1)
    return fact, dim, extra


def _star_query(n_extra, dim_filters=(None, None, None, None)):
    q = dict(W.q_lowcard(), dim_filter=dim_filters[0])
    q["extra_joins"] = [dict(fact_col=f"fk{j + 2}", dim_col="pk", dim_filter=dim_filters[j + 1])
                        for j in range(n_extra)]
    bands = [(f"dim{j + 1}", "band", 2) for j in range(n_extra)]
    q["group"] = ([("fact", "flag", 2)] if n_extra < 3 else []) + [("dim", "attr", 5)] + bands   # at most 4 fields
    return q


@pytest.mark.parametrize("seed,n_extra,filters", [
    (40, 1, (None, None)),
    (41, 2, (None, dict(col="attr", lo=0, hi=12), None)),
    (42, 3, (dict(col="attr", lo=5, hi=20), None, dict(col="band", lo=1, hi=2), dict(col="attr", lo=0, hi=0))),
    (43, 2, (None, dict(col="attr", lo=30, hi=40), None)),       # a dimension admits nothing: empty result
])
def test_star_join_matches_bruteforce(seed, n_extra, filters):
    fact, dim, extra = _star_tiny(seed, 700, [60, 40, 30, 20][:n_extra + 1], [80, 50, 35, 25][:n_extra + 1])
    q = _star_query(n_extra, filters)
    ref = bruteforce.evaluate(fact, dim, q, extra)
    got = oracle.run_query(fact, dim, q, extra)
    assert got.n_groups == len(ref)
    for g, (key, count, sums, avgs) in enumerate(ref):
        assert int(got.keys[g]) == key and int(got.counts[g]) == count
        for a, ag in enumerate(q["aggs"]):
            assert got.sum_int(g, a) == sums[a]
            if ag[0] == "avg":
                assert got.avgs[g, a] == avgs[a]
    if filters[-1] is not None and filters[-1]["lo"] > 24:
        assert got.n_groups == 0


def test_star_join_field_equals_derived_fact_column():
    """A dimension whose attribute is a function of its key: grouping by that
    attribute through the join equals grouping by the function of the foreign
    key computed on the fact side, restricted to rows that have a partner."""
    fact, dim, extra = _star_tiny(44, 3000, [200, 500], [200, 700])
    extra[0]["band"] = (extra[0]["pk"] % 4).astype(np.uint8)
    q = _star_query(1)
    got = oracle.run_query(fact, dim, q, extra)
    f2 = {k: v.copy() for k, v in fact.items()}
    hit = f2["fk2"] < 500                                 # keys 0..499 exist in the second dimension
    f2["date"] = np.where(hit, f2["date"], W.N_DAYS + 10).astype(np.int32)   # drop the misses by the filter
    f2["band2"] = (f2["fk2"] % 4).astype(np.uint8)
    q2 = dict(W.q_lowcard(), group=[("fact", "flag", 2), ("dim", "attr", 5), ("fact", "band2", 2)])
    want = oracle.run_query(f2, dim, q2)
    assert np.array_equal(got.keys, want.keys) and np.array_equal(got.counts, want.counts)
    assert np.array_equal(got.sums, want.sums)


def test_star_join_order_of_dimensions_is_irrelevant():
    fact, dim, extra = _star_tiny(45, 2500, [90, 70, 50], [100, 80, 60])
    q = _star_query(2, (dict(col="attr", lo=0, hi=15), None, dict(col="band", lo=0, hi=2)))
    base = oracle.run_query(fact, dim, q, extra)
    # the second further dimension as the first join and the first join as a further one
    fact_sw = dict(fact, fk=fact["fk3"], fk3=fact["fk"].astype(np.int64))
    q_sw = dict(q, dim_filter=q["extra_joins"][1]["dim_filter"])
    q_sw["extra_joins"] = [q["extra_joins"][0], dict(fact_col="fk3", dim_col="pk", dim_filter=q["dim_filter"])]
    q_sw["group"] = [("fact", "flag", 2), ("dim2", "attr", 5), ("dim1", "band", 2), ("dim", "band", 2)]
    sw = oracle.run_query(fact_sw, extra[1], q_sw, [extra[0], dim])
    # the fields land in the same key bits, so the results are identical
    assert np.array_equal(base.keys, sw.keys) and np.array_equal(base.counts, sw.counts)
    assert np.array_equal(base.sums, sw.sums)


def _fanout_tiny(seed, n_fact, n_keys, span):
    """A dimension whose keys repeat: key k appears 1 + (k mod 4) times (some
    rows with different attributes), shuffled."""
    fact, _ = _tiny(seed, n_fact, 0, span)
    reps = 1 + np.arange(n_keys) % 4
    pk = np.repeat(np.arange(n_keys, dtype=np.int32), reps)
    perm = datagen.fill(3000 + seed, 1, datagen.PERM, np.int64, len(pk), b=len(pk))
    dim = dict(pk=pk[perm], attr=datagen.uniform(3000 + seed, 2, np.int32, len(pk), 0, 24))
    return fact, dim


@pytest.mark.parametrize("seed,dflt", [(70, None), (71, dict(col="attr", lo=4, hi=15)), (72, dict(col="attr", lo=30, hi=31))])
def test_fanout_join_matches_bruteforce(seed, dflt):
    fact, dim = _fanout_tiny(seed, 800, 60, 75)
    q = dict(W.q_lowcard(), join=dict(fact_col="fk", dim_col="pk", many=True), dim_filter=dflt)
    got = _check_against_brute(fact, dim, q)
    partners = {}
    for k, a in zip(dim["pk"], dim["attr"]):
        if dflt is None or dflt["lo"] <= a <= dflt["hi"]:
            partners[int(k)] = partners.get(int(k), 0) + 1
    want = sum(partners.get(int(fk), 0) for fk, dt in zip(fact["fk"], fact["date"]) if dt <= W.CUTOFF_98)
    assert int(got.counts.sum()) == want
    if dflt is None:   # without fan-out the repeated keys are an error
        with pytest.raises(oracle.OracleError) as e:
            oracle.run_query(fact, dim, dict(q, join=dict(fact_col="fk", dim_col="pk")))
        assert e.value.status == "dup_key"


def test_fanout_of_identical_rows_doubles_everything():
    """Every dimension row present twice: each group's count and sums are
    exactly twice those of the join with unique keys."""
    fact, dim = _tiny(73, 5000, 300, 350, signed=True)
    twice = {k: np.concatenate([v, v]) for k, v in dim.items()}
    q = W.q_lowcard()
    one = oracle.run_query(fact, dim, q)
    two = oracle.run_query(fact, twice, dict(q, join=dict(q["join"], many=True)))
    assert np.array_equal(one.keys, two.keys)
    assert np.array_equal(2 * one.counts, two.counts)
    for g in range(one.n_groups):
        for a in (0, 1, 2):
            assert two.sum_int(g, a) == 2 * one.sum_int(g, a)


def test_fanout_with_a_further_dimension():
    fact, dim = _fanout_tiny(74, 600, 40, 50)
    _, _, extra = _star_tiny(74, 600, [40, 30], [50, 40])
    fact["fk2"] = datagen.uniform(4074, 5, np.int64, 600, 0, 39)
    q = dict(W.q_lowcard(), join=dict(fact_col="fk", dim_col="pk", many=True),
             extra_joins=[dict(fact_col="fk2", dim_col="pk", dim_filter=dict(col="band", lo=0, hi=2))])
    q["group"] = [("fact", "flag", 2), ("dim", "attr", 5), ("dim1", "band", 2)]
    ref = bruteforce.evaluate(fact, dim, q, extra)
    got = oracle.run_query(fact, dim, q, extra)
    assert got.n_groups == len(ref)
    for g, (key, count, sums, _) in enumerate(ref):
        assert int(got.keys[g]) == key and int(got.counts[g]) == count
        for a in range(len(q["aggs"])):
            assert got.sum_int(g, a) == sums[a]


def _modular_closed_form(n_fact, n_dim):
    """Per-group (count, SUM qty, SUM price*(100-disc), SUM disc) on the
    modular dataset, from arithmetic series.  Row i has flag = i mod 3,
    status = i mod 2, attr = (i mod n_dim) mod 25 = i mod 25 (25 | n_dim), so
    the group is the residue r = i mod 150 and holds T = n_fact / 150 rows
    i = r + 150 t.  qty = (i mod 50)*100 + 100 is constant on the group;
    (i mod 7, i mod 11) runs over all 77 pairs once per 77 steps of t since
    150 is invertible mod 7 and mod 11; disc = i mod 11 sums to 55 per 11 steps."""
    assert n_fact % (150 * 77) == 0 and n_dim % 25 == 0
    T = n_fact // 150
    price_sum = sum(1000 * a + 90_000 for a in range(7))       # 651000
    mult_sum = sum(100 - b for b in range(11))                  # 1045
    out = {}
    for r in range(150):
        key = ((r % 3) << 6) | ((r % 2) << 5) | (r % 25)
        out[key] = (T, T * ((r % 50) * 100 + 100), (T // 77) * price_sum * mult_sum, (T // 11) * 55)
    return out


@pytest.mark.parametrize("n_fact,n_dim", [(11550, 200), (23100, 1000), (150 * 77 * 6, 25)])
def test_modular_closed_form(n_fact, n_dim):
    wl = W.modular(n_fact, n_dim)
    got = oracle.run(wl)
    want = _modular_closed_form(n_fact, n_dim)
    assert got.n_groups == 150
    assert sorted(want) == [int(k) for k in got.keys]
    for g, key in enumerate(got.keys):
        cnt, s_qty, s_rev, s_disc = want[int(key)]
        assert int(got.counts[g]) == cnt
        assert got.sum_int(g, 0) == s_qty
        assert got.sum_int(g, 1) == s_rev
        assert got.sum_int(g, 2) == cnt
        assert got.sum_int(g, 3) == s_disc
        assert got.avgs[g, 3] == s_disc / cnt == 5.0


def _torch_int64(fact, dim, query):
    """Second evaluation with PyTorch CPU int64 ops: searchsorted join,
    unique/index_add_ grouping.  Valid while every sum fits in int64."""
    import torch
    f = {k: torch.from_numpy(np.asarray(v).astype(np.int64)) for k, v in fact.items()}
    d = {k: torch.from_numpy(np.asarray(v).astype(np.int64)) for k, v in dim.items()}
    flt = query["filter"]
    keep = (f[flt["col"]] >= flt["lo"]) & (f[flt["col"]] <= flt["hi"])
    dflt = query.get("dim_filter")
    if dflt is not None:   # drop the dimension rows the predicate rejects
        dk = (d[dflt["col"]] >= dflt["lo"]) & (d[dflt["col"]] <= dflt["hi"])
        d = {k: v[dk] for k, v in d.items()}
    pk_sorted, order = torch.sort(d[query["join"]["dim_col"]])
    fk = f[query["join"]["fact_col"]]
    pos = torch.searchsorted(pk_sorted, fk).clamp(max=pk_sorted.numel() - 1)
    hit = pk_sorted[pos] == fk
    keep &= hit
    drow = order[pos]
    idx = torch.nonzero(keep).flatten()
    key = torch.zeros(idx.numel(), dtype=torch.int64)
    for side, col, bits in query["group"]:
        v = f[col][idx] if side == "fact" else d[col][drow[idx]]
        key = (key << bits) | v
    uniq, inv = torch.unique(key, return_inverse=True)
    cols = []
    for ag in query["aggs"]:
        if ag[0] in ("sum", "avg"):
            t = f[ag[1]][idx]
        elif ag[0] == "sum_mul_sub":
            t = f[ag[1]][idx] * (ag[2] - f[ag[3]][idx])
        else:
            t = torch.ones_like(idx)
        acc = torch.zeros(uniq.numel(), dtype=torch.int64).index_add_(0, inv, t)
        cols.append(acc)
    cnt = torch.zeros(uniq.numel(), dtype=torch.int64).index_add_(0, inv, torch.ones_like(idx))
    return uniq.numpy(), cnt.numpy(), [c.numpy() for c in cols]


@pytest.mark.parametrize("maker", ["config1", "config2a", "config2a_dimfilter"])
def test_second_oracle_torch_int64(maker):
    if maker == "config1":
        wl = W.config1(n_fact=300_000, n_dim=10_000)
    else:
        wl = W.config2("a", n_fact=300_000, n_dim=50_000)
    if maker.endswith("dimfilter"):
        wl.query["dim_filter"] = dict(col="attr", lo=3, hi=7)
    got = oracle.run(wl)
    keys, cnt, sums = _torch_int64(wl.fact, wl.dim, wl.query)
    assert np.array_equal(got.keys.astype(np.int64), keys)
    assert np.array_equal(got.counts, cnt)
    for a in range(len(wl.query["aggs"])):
        assert np.all(got.sums[:, a, 1].astype(np.int64) == 0)     # all sums are small here
        assert np.array_equal(got.sums[:, a, 0].astype(np.int64), sums[a])


def test_invariants_config1_small():
    wl = W.config1(n_fact=200_000, n_dim=10_000)
    got = oracle.run(wl)
    f = wl.fact
    passing = int((f["date"] <= W.CUTOFF_98).sum())          # every fk matches a pk
    assert int(got.counts.sum()) == passing
    assert got.n_groups == 150
    # grouped sums add up to the ungrouped query's sums
    q0 = dict(wl.query, group=[])
    tot = oracle.run_query(f, wl.dim, q0)
    assert tot.n_groups == 1 and int(tot.keys[0]) == 0
    for a in range(4):
        assert sum(got.sum_int(g, a) for g in range(got.n_groups)) == tot.sum_int(0, a)
    # AVG * COUNT reproduces SUM(disc) within 1e-15 relative
    for g in range(got.n_groups):
        s, c = got.sum_int(g, 3), int(got.counts[g])
        assert got.avgs[g, 3] == float(s) / float(c)
        assert abs(got.avgs[g, 3] * c - s) <= 1e-15 * abs(s) + 1e-300


def test_row_order_independence():
    wl = W.config1(n_fact=50_000, n_dim=2_000)
    base = oracle.run(wl)
    perm = datagen.fill(77, 0, datagen.PERM, np.int64, wl.n_fact, b=wl.n_fact)
    fact = {k: v[perm] for k, v in wl.fact.items()}
    dperm = datagen.fill(78, 0, datagen.PERM, np.int64, wl.n_dim, b=wl.n_dim)
    dim = {k: v[dperm] for k, v in wl.dim.items()}
    other = oracle.run_query(fact, dim, wl.query)
    assert np.array_equal(base.keys, other.keys)
    assert np.array_equal(base.counts, other.counts)
    assert np.array_equal(base.sums, other.sums)
    assert np.array_equal(base.avgs, other.avgs)


def test_int128_wraps_like_fixed_width_sum():
    """Terms near 2^126: the exact sum leaves int128, and the oracle must agree
    with the Python big-int sum reduced modulo 2^128."""
    n = 16
    fact = dict(a=np.full(n, I64_MAX - 3, np.int64), b=np.full(n, I64_MIN + 5, np.int64),
                g=np.zeros(n, np.uint8))
    q = dict(filter=None, join=None, group=[("fact", "g", 1)],
             aggs=[("sum_mul_sub", "a", I64_MAX, "b"), ("sum", "b")])
    got = oracle.run_query(fact, None, q)
    term = (I64_MAX - 3) * (I64_MAX - (I64_MIN + 5))
    exact = n * term
    wrapped = exact % (1 << 128)
    wrapped = wrapped - (1 << 128) if wrapped >= 1 << 127 else wrapped
    assert got.sum_int(0, 0) == wrapped
    assert got.sum_int(0, 1) == n * (I64_MIN + 5)        # below -2^63: needs the high word


def test_i128_to_double_is_correctly_rounded():
    vals = [0, 1, -1, (1 << 53) + 1, (1 << 64) + 1, -(1 << 100) - 12345, (1 << 127) - 1, -(1 << 127)]
    # values right at and beside rounding ties at several magnitudes
    for e in (54, 60, 64, 70, 100, 126):
        base = 1 << e
        ulp = 1 << (e - 52)
        for off in (ulp // 2 - 1, ulp // 2, ulp // 2 + 1, 3 * ulp // 2):
            vals += [base + off, -(base + off)]
    raw = datagen.fill(5, 5, datagen.RAW64, np.int64, 400)
    for i in range(0, 400, 2):
        v = (int(raw[i]) << 64) | (int(raw[i + 1]) & ((1 << 64) - 1))
        vals.append(v >> (i % 100))
    for v in vals:
        assert oracle.i128_to_double(v) == float(v), v
    assert math.isfinite(oracle.i128_to_double(-(1 << 127)))
