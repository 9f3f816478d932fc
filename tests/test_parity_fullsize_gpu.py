"""The star workload at full size (60M fact rows, 2M-row dimension, Zipf
foreign keys) in the launch configuration the benchmark times: the
low-cardinality and 1%-selective queries against the full oracle, the ~98%
high-cardinality query against per-group oracle samples and invariants."""
import numpy as np
import pytest

import oracle
from datagen import workloads as W
from paper_2508_05029_gb300 import theseus as T
from tests.helpers import assert_matches_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def star():
    from paper_2508_05029_gb300 import build
    import torch
    build.build()
    fact, dim = W.config2_tables()
    eng = T.Engine()
    ft = eng.table_from_torch({k: torch.from_numpy(v).cuda() for k, v in fact.items()})
    dt = eng.table_from_torch({k: torch.from_numpy(v).cuda() for k, v in dim.items()})
    yield eng, fact, dim, ft, dt
    ft.destroy()
    dt.destroy()
    eng.close()


def _run(star, query):
    eng, fact, dim, ft, dt = star
    p = eng.plan(ft, dt, query)
    try:
        return p.execute()
    finally:
        p.destroy()


@pytest.mark.parametrize("which", ["a", "b"])
def test_full_oracle(star, which):
    _, fact, dim, _, _ = star
    q = W.q_lowcard() if which == "a" else W.q_highcard(W.config2_range_lo(), W.config2_range_lo() + W.RANGE_1PCT)
    ref = oracle.run_query(fact, dim, q)
    with _run(star, q) as res:
        assert_matches_oracle(res, ref, q["aggs"])
    if which == "a":
        assert ref.n_groups == 150
    else:
        assert 400_000 < ref.n_groups < 800_000


def test_highcard_98pct_samples_and_invariants(star):
    _, fact, dim, _, _ = star
    q = W.q_highcard(0, W.CUTOFF_98)
    with _run(star, q) as res:
        keys, counts, sums = res.keys(), res.counts(), res.sum_words(0)
    assert np.all(np.diff(keys.astype(np.uint64)) > 0)
    passing = int((fact["date"] <= W.CUTOFF_98).sum())      # every fk has a partner
    assert int(counts.sum()) == passing
    assert 14_000_000 < keys.size <= 15_000_000
    # exact grand total against the oracle's ungrouped query
    tot = oracle.run_query(fact, dim, dict(q, group=[]))
    total = int(np.sum(sums[:, 0].astype(object))) + (int(np.sum(sums[:, 1].astype(np.int64).astype(object))) << 64)
    assert total == tot.sum_int(0, 0)
    # sampled groups: the rows of an order key are the four rows 4j..4j+3
    rng_rows = np.linspace(0, len(fact["okey"]) - 4, 200).astype(np.int64) & ~3
    for r0 in rng_rows:
        sub = {k: v[r0:r0 + 4] for k, v in fact.items()}
        ref = oracle.run_query(sub, dim, q)
        for g in range(ref.n_groups):
            i = np.searchsorted(keys, ref.keys[g])
            assert keys[i] == ref.keys[g]
            assert counts[i] == ref.counts[g]
            assert int(sums[i, 0]) == int(ref.sums[g, 0, 0]) and int(sums[i, 1]) == int(ref.sums[g, 0, 1])
