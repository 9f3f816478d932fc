"""The seeded input generator: determinism, row-indexability, ranges."""
import numpy as np

import datagen
from datagen import workloads as W


def test_row_ranges_regenerate_independently():
    full = datagen.uniform(11, 3, np.int64, 10_000, -7, 1_000)
    part = datagen.uniform(11, 3, np.int64, 1_000, -7, 1_000, row0=4_321)
    assert np.array_equal(full[4_321:5_321], part)
    assert full.min() >= -7 and full.max() <= 1_000
    assert np.array_equal(full, datagen.uniform(11, 3, np.int64, 10_000, -7, 1_000))
    assert not np.array_equal(full, datagen.uniform(12, 3, np.int64, 10_000, -7, 1_000))


def test_permutations_are_bijections():
    for n in (1, 2, 3, 1000, 4097, 65_536, 1_000_003):
        p = datagen.fill(5, 9, datagen.PERM, np.int64, n, b=n)
        assert np.array_equal(np.sort(p), np.arange(n))
    p = datagen.fill(5, 9, datagen.PERM, np.int64, 1000, b=1000)
    assert (p != np.arange(1000)).mean() > 0.9


def test_raw64_unique_and_zipf_skew():
    raw = datagen.fill(1, 1, datagen.RAW64, np.int64, 1_000_000)
    assert np.unique(raw).size == raw.size
    assert np.array_equal(datagen.raw_at(1, 1, np.array([5, 999_999, 0])), raw[[5, 999_999, 0]])
    cdf = datagen.zipf_cdf(0.8, 100_000)
    idx = datagen.index(3, 3, 100_000, 500_000, cdf=cdf)
    counts = np.bincount(idx, minlength=100_000)
    top = np.sort(counts)[::-1]
    assert top[0] / idx.size > 0.01             # hottest rank ~1/H(0.8) of the mass
    assert top[0] > 20 * np.median(counts)


def test_config_shapes():
    wl = W.config1(n_fact=100_000, n_dim=10_000)
    f = wl.fact
    assert f["fk"].dtype == np.int32 and f["qty"].dtype == np.int64 and f["flag"].dtype == np.uint8
    assert f["qty"].min() >= 100 and f["qty"].max() <= 5000 and (f["qty"] % 100 == 0).all()
    assert f["price"].min() >= 90_000 and f["price"].max() <= 10_500_000
    assert f["disc"].min() >= 0 and f["disc"].max() <= 10
    assert 0.975 < (f["date"] <= W.CUTOFF_98).mean() < 0.985
    fact, dim = W.config2_tables(n_fact=400_000, n_dim=100_000)
    assert np.unique(dim["pk"]).size == 100_000
    assert np.isin(fact["fk"], dim["pk"]).all()
    assert np.unique(fact["okey"]).size == 100_000
    sizes = W.config4_sizes()
    assert sizes["fact"].min() >= 10_000 and sizes["fact"].max() <= 50_000_000
    assert 1e8 < sizes["fact"].sum() < 1e9


def test_star_dimension_and_foreign_keys():
    """A further star dimension: unique sparse keys, attributes in range, and
    every generated foreign key names one of its rows (regenerated by row)."""
    from datagen import workloads as W
    seed = W.SEEDS[2] + 100
    d = W.star_dim(50_000, seed)
    assert len(np.unique(d["pk"])) == 50_000
    assert d["attr"].min() >= 0 and d["attr"].max() <= 24 and d["band"].max() <= 3
    fk = W.star_fk(200_000, 50_000, seed)
    assert np.isin(fk, d["pk"]).all()
    # uniform over the rows: every row is hit about 4 times
    _, hits = np.unique(fk, return_counts=True)
    assert len(hits) > 0.97 * 50_000 and hits.max() < 20
    # row ranges regenerate independently, and another dimension index gives other keys
    assert np.array_equal(W.star_dim(50_000, seed)["pk"][:100], d["pk"][:100])
    assert not np.isin(W.star_dim(1_000, seed, j=1)["pk"], d["pk"]).any()


def test_sparse_star_keys_unique_and_joinable():
    """The sparse-key star tables: int64 dimension keys, all distinct and far
    from dense, and every foreign key one of them."""
    fact, dim = W.config2_tables(n_fact=50_000, n_dim=4_000, sparse_keys=True)
    pk = dim["pk"]
    assert pk.dtype == np.int64 and fact["fk"].dtype == np.int64
    assert np.unique(pk).size == pk.size
    assert int(pk.max()) - int(pk.min()) > 1000 * pk.size
    assert np.isin(fact["fk"], pk).all()
