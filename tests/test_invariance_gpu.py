"""Metamorphic checks of the CUDA path: permuting fact or dimension rows, and
changing the page size and batch size of paged tables, leave every group's
result unchanged (and equal to the oracle's)."""
import numpy as np
import pytest

import datagen
import oracle
from datagen import workloads as W
from paper_2508_05029_gb300 import theseus as T
from tests.helpers import assert_matches_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2508_05029_gb300 import build
    build.build()


def _run(eng, fact, dim, q, placement):
    ft = eng.table_from_numpy(fact, placement=placement)
    dt = eng.table_from_numpy(dim, placement=placement)
    p = eng.plan(ft, dt, q)
    try:
        r = p.execute()
        out = (r.keys(), r.counts(), [r.sum_words(a) for a in (0, 1, 3)], r.avg(3))
        r.free()
        return out
    finally:
        p.destroy()
        ft.destroy()
        dt.destroy()


def _same(x, y):
    assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) and np.array_equal(x[3], y[3])
    for a, b in zip(x[2], y[2]):
        assert np.array_equal(a, b)


def test_row_permutations_change_nothing():
    wl = W.config2("a", n_fact=1_000_003, n_dim=50_000)
    perm = datagen.fill(91, 0, datagen.PERM, np.int64, wl.n_fact, b=wl.n_fact)
    dperm = datagen.fill(92, 0, datagen.PERM, np.int64, wl.n_dim, b=wl.n_dim)
    fact_p = {k: v[perm] for k, v in wl.fact.items()}
    dim_p = {k: v[dperm] for k, v in wl.dim.items()}
    e = T.Engine(page_bytes=8 << 20, n_pages=64, batch_rows=1 << 20)
    try:
        base = _run(e, wl.fact, wl.dim, wl.query, T.TP_DEVICE)
        _same(base, _run(e, fact_p, wl.dim, wl.query, T.TP_DEVICE))
        _same(base, _run(e, wl.fact, dim_p, wl.query, T.TP_DEVICE))
        _same(base, _run(e, fact_p, dim_p, wl.query, T.TP_DEVICE))
        ref = oracle.run(wl)
        assert np.array_equal(base[0], ref.keys) and np.array_equal(base[1], ref.counts)
    finally:
        e.close()


@pytest.mark.parametrize("page_mb,batch_rows", [(1, 10_000), (4, 123_457), (16, 1 << 20)])
def test_page_and_batch_sizes_change_nothing(page_mb, batch_rows):
    wl = W.config2("a", n_fact=700_001, n_dim=40_000)
    ref = oracle.run(wl)
    rows = wl.n_fact * 34 + wl.n_dim * 8
    n_pages = int(2 * rows // (page_mb << 20)) + 2 * (wl.n_fact // batch_rows + 2) + 16
    e = T.Engine(page_bytes=page_mb << 20, n_pages=n_pages, batch_rows=batch_rows)
    try:
        ft = e.table_from_numpy(wl.fact, placement=T.TP_HOST_PAGES)
        dt = e.table_from_numpy(wl.dim, placement=T.TP_HOST_PAGES)
        p = e.plan(ft, dt, wl.query)
        with p.execute() as r:
            assert_matches_oracle(r, ref, wl.query["aggs"])
        p.destroy()
        ft.destroy()
        dt.destroy()
    finally:
        e.close()
