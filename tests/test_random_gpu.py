"""Random query shapes through the CUDA path: seeded tiny star schemas
(filters, predicates, fan-out, further dimensions, group fields from any
table, every aggregate kind) on random kernel paths, placements and lookahead
settings; each result equals the oracle's, and each error is the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2508_05029_gb300 import theseus as T
from tests.helpers import assert_matches_oracle

pytestmark = pytest.mark.gpu

FLAGS = [0, T.TP_FLAG_NO_JIT, T.TP_FLAG_NO_STAGED, T.TP_FLAG_NO_DIRECT_JOIN, T.TP_FLAG_NO_DIRECT_AGG,
         T.TP_FLAG_EXACT_ONLY]


def _case(seed):
    rng = np.random.default_rng(0xC0FFEE + seed)
    n_fact = int(rng.integers(0, 5000))
    n_dim = int(rng.integers(0, 300))
    n_x = int(rng.integers(0, 3))
    many = bool(rng.integers(0, 2))
    ints = lambda n, lo, hi, dt=np.int64: rng.integers(lo, hi + 1, n).astype(dt)
    fact = dict(fk=ints(n_fact, -2, 330, np.int32), a=ints(n_fact, -10**6, 10**6), b=ints(n_fact, -50, 50),
                f=ints(n_fact, 0, 3, np.uint8), d=ints(n_fact, 0, 99, np.int32))
    # unique keys unless fan-out (then about half the keys repeat)
    pk = rng.permutation(n_dim).astype(np.int32) if not many else ints(n_dim, 0, max(1, n_dim // 2), np.int32)
    dim = dict(pk=pk, attr=ints(n_dim, 0, 5, np.int32))
    extra = []
    q = dict(join=dict(fact_col="fk", dim_col="pk", many=many), extra_joins=[])
    for j in range(n_x):
        n = int(rng.integers(0, 100))
        extra.append(dict(pk=rng.permutation(n).astype(np.int64) * 3, band=ints(n, 0, 3, np.uint8)))
        fact[f"fk{j + 2}"] = ints(n_fact, 0, 3 * n + 5)
        xj = dict(fact_col=f"fk{j + 2}", dim_col="pk")
        if rng.integers(0, 2):
            xj["dim_filter"] = dict(col="band", lo=0, hi=int(rng.integers(0, 4)))
        q["extra_joins"].append(xj)
    if rng.integers(0, 2):
        lo = int(rng.integers(0, 100))
        q["filter"] = dict(col="d", lo=lo, hi=lo + int(rng.integers(0, 100)))
    if rng.integers(0, 2):
        lo = int(rng.integers(0, 6))
        q["dim_filter"] = dict(col="attr", lo=lo, hi=lo + int(rng.integers(0, 4)))
    fields = [("fact", "f", 2), ("dim", "attr", 3), ("fact", "d", 7)] + [(f"dim{j + 1}", "band", 2)
                                                                          for j in range(n_x)]
    pick = rng.permutation(len(fields))[: int(rng.integers(0, 5))]
    q["group"] = [fields[i] for i in pick]
    aggs = [("sum", "a"), ("avg", "b"), ("count",), ("sum_mul_sub", "a", 7, "b"), ("avg", "a")]
    q["aggs"] = [aggs[i] for i in rng.integers(0, len(aggs), int(rng.integers(1, 5)))]
    opts = dict(flags=FLAGS[int(rng.integers(0, len(FLAGS)))],
                placement=[T.TP_DEVICE, T.TP_HOST_PAGES][int(rng.integers(0, 2))],
                lip=[T.TP_LIP_AUTO, T.TP_LIP_ON, T.TP_LIP_OFF][int(rng.integers(0, 3))])
    return fact, dim, extra, q, opts


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_05029_gb300 import build
    build.build()


@pytest.mark.parametrize("seed", range(48))
def test_random_query_matches_oracle(seed):
    fact, dim, extra, q, opts = _case(seed)
    try:
        ref = oracle.run_query(fact, dim, q, extra)
        want_err = None
    except oracle.OracleError as e:
        ref, want_err = None, e.status
    e = T.Engine(page_bytes=1 << 20, n_pages=64, batch_rows=1024, flags=opts["flags"])
    try:
        tabs = [e.table_from_numpy(t, placement=opts["placement"]) for t in [fact, dim] + extra]
        p = e.plan(tabs[0], tabs[1], q, extra_dims=tabs[2:], lip=opts["lip"])
        try:
            if want_err is not None:
                with pytest.raises(T.TPError) as err:
                    p.execute()
                assert err.value.status == want_err
            else:
                with p.execute() as r:
                    assert_matches_oracle(r, ref, q["aggs"])
        finally:
            p.destroy()
            for t in tabs:
                t.destroy()
    finally:
        e.close()
