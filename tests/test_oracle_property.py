"""Property pin of the oracle: on random tiny star schemas and random query
shapes (filters, predicates, group fields from any table, every aggregate kind,
fan-out, further dimensions) the oracle equals the nested-loop brute force,
including which inputs are errors."""
import numpy as np
import pytest

import oracle
from tests import bruteforce

hypothesis = pytest.importorskip("hypothesis")
st = hypothesis.strategies


@st.composite
def star_case(draw):
    n_fact = draw(st.integers(0, 40))
    n_dim = draw(st.integers(0, 12))
    n_x = draw(st.integers(0, 2))
    ints = lambda n, lo, hi: np.array(draw(st.lists(st.integers(lo, hi), min_size=n, max_size=n)), np.int64)
    fact = dict(fk=ints(n_fact, -2, 14), a=ints(n_fact, -1000, 1000), b=ints(n_fact, -50, 50),
                f=ints(n_fact, 0, 3), d=ints(n_fact, 0, 9))
    dim = dict(pk=ints(n_dim, -2, 14), attr=ints(n_dim, 0, 5))
    extra = []
    for j in range(n_x):
        n = draw(st.integers(0, 8))
        extra.append(dict(pk=ints(n, 0, 9), band=ints(n, 0, 3)))
        fact[f"fk{j + 2}"] = ints(n_fact, 0, 11)
    many = draw(st.booleans())
    q = dict(join=dict(fact_col="fk", dim_col="pk", many=many))
    if draw(st.booleans()):
        lo = draw(st.integers(0, 9))
        q["filter"] = dict(col="d", lo=lo, hi=lo + draw(st.integers(0, 9)))
    if draw(st.booleans()):
        lo = draw(st.integers(0, 5))
        q["dim_filter"] = dict(col="attr", lo=lo, hi=lo + draw(st.integers(0, 3)))
    q["extra_joins"] = []
    for j in range(n_x):
        xj = dict(fact_col=f"fk{j + 2}", dim_col="pk")
        if draw(st.booleans()):
            xj["dim_filter"] = dict(col="band", lo=0, hi=draw(st.integers(0, 3)))
        q["extra_joins"].append(xj)
    fields = [("fact", "f", 2), ("dim", "attr", 3)] + [(f"dim{j + 1}", "band", 2) for j in range(n_x)]
    q["group"] = draw(st.lists(st.sampled_from(fields), max_size=4, unique=True))
    aggs = [("sum", "a"), ("avg", "b"), ("count",), ("sum_mul_sub", "a", 7, "b")]
    q["aggs"] = draw(st.lists(st.sampled_from(aggs), min_size=1, max_size=4))
    return fact, dim, extra, q


@hypothesis.settings(max_examples=300, deadline=None)
@hypothesis.given(star_case())
def test_oracle_equals_brute_force_on_random_star_queries(case):
    fact, dim, extra, q = case
    try:
        ref = bruteforce.evaluate(fact, dim, q, extra)
    except ValueError as err:
        with pytest.raises(oracle.OracleError) as e:
            oracle.run_query(fact, dim, q, extra)
        assert e.value.status == str(err)
        return
    got = oracle.run_query(fact, dim, q, extra)
    assert got.n_groups == len(ref)
    for g, (key, count, sums, avgs) in enumerate(ref):
        assert int(got.keys[g]) == key and int(got.counts[g]) == count
        for a, ag in enumerate(q["aggs"]):
            assert got.sum_int(g, a) == sums[a]
            if ag[0] == "avg":
                assert got.avgs[g, a] == avgs[a]
