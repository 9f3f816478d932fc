"""Shared test helpers: compare a GPU result with the oracle's."""
import numpy as np

AVG_RTOL = 1e-15   # AVG: exact sum / count in FP64, within 1e-15 relative


def assert_matches_oracle(res, ref, aggs):
    """Keys, counts and 128-bit sums bit-exact; AVG within AVG_RTOL (and, since
    both sides round the exact sum once and divide once, bit-identical)."""
    assert res.n_groups == ref.n_groups, (res.n_groups, ref.n_groups)
    if ref.n_groups == 0:
        return
    assert np.array_equal(res.keys(), ref.keys)
    assert np.array_equal(res.counts(), ref.counts)
    for a, ag in enumerate(aggs):
        if ag[0] == "count":
            continue
        got = res.sum_words(a)
        assert np.array_equal(got[:, 0], ref.sums[:, a, 0]), f"agg {a} low words differ"
        assert np.array_equal(got[:, 1], ref.sums[:, a, 1]), f"agg {a} high words differ"
        if ag[0] == "avg":
            av = res.avg(a)
            want = ref.avgs[:, a]
            rel = np.abs(av - want) / np.maximum(np.abs(want), np.finfo(np.float64).tiny)
            assert float(rel.max()) <= AVG_RTOL
            assert np.array_equal(av, want)
