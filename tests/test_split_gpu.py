"""Split-and-retry of a global aggregation (Section 3.3.2: a task that runs out
of memory is retried and divided up): when the aggregation table of a
many-group query cannot be reserved, the packed group key range is halved
until each range's table fits, one pass per range.  Results must equal the
oracle's whatever the budget; a budget too small for any split fails with
TP_E_BUDGET, never with a wrong answer."""
import numpy as np
import pytest

import oracle
from datagen import workloads as W
from paper_2508_05029_gb300 import theseus as T
from tests.helpers import assert_matches_oracle

pytestmark = pytest.mark.gpu

N_FACT, N_DIM = 2_000_000, 50_000


@pytest.fixture(scope="module")
def data():
    from paper_2508_05029_gb300 import build
    build.build()
    fact, dim = W.config2_tables(n_fact=N_FACT, n_dim=N_DIM)      # 500k order keys, 4 rows each
    q = W.q_highcard(0, W.CUTOFF_98)
    q = dict(q, aggs=q["aggs"] + [("avg", "qty")])
    return fact, dim, q, oracle.run_query(fact, dim, q)


def _run(flags, budget, fact, dim, q, ref, **kw):
    """Runs q under the budget and checks it against the oracle; returns
    (extra split passes, peak reservation), or None when the budget refused
    it."""
    e = T.Engine(page_bytes=2 << 20, n_pages=256, batch_rows=250_000, flags=flags)
    try:
        e.set_budget(budget)
        ft = e.table_from_numpy(fact, placement=T.TP_HOST_PAGES)
        dt = e.table_from_numpy(dim, placement=T.TP_HOST_PAGES)
        p = e.plan(ft, dt, q, **kw)
        try:
            s0 = e.stats()["agg_split_passes"]
            try:
                res = p.execute()
            except T.TPError as err:
                assert err.status == "budget", err
                return None
            with res:
                assert_matches_oracle(res, ref, q["aggs"])
            st = e.stats()
            return st["agg_split_passes"] - s0, st["peak_reserved"]
        finally:
            p.destroy()
            ft.destroy()
            dt.destroy()
    finally:
        e.close()


@pytest.mark.parametrize("flags,kw", [
    (0, {}),                                          # direct-addressed ranges
    (T.TP_FLAG_NO_DIRECT_AGG, {}),                    # hashed ranges
    (T.TP_FLAG_NO_DIRECT_AGG, dict(expected_groups=1000)),   # overflow retries that end in a split
], ids=["direct", "hashed", "underestimate"])
def test_split_matches_oracle_at_every_budget(data, flags, kw):
    fact, dim, q, ref = data
    passes, peak = _run(flags, 4 << 30, fact, dim, q, ref, **kw)
    assert passes == 0                                # room for everything: one pass
    split_ok = 0
    for frac in (0.9, 0.8, 0.7, 0.6, 0.55, 0.5):
        r = _run(flags, int(peak * frac), fact, dim, q, ref, **kw)
        print(f"budget {frac:.2f} x {peak >> 20} MiB: {r}")
        split_ok += r is not None and r[0] > 0
    assert split_ok >= 2                              # at least two budgets ran split, both correct
