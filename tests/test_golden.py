"""Golden fixtures (tests/golden/*.txt, written by tests/golden/make_golden.py
from the oracle alone): the oracle must keep reproducing them, the modular
one must agree with its arithmetic-series closed form, and the CUDA path must
reproduce them bit for bit."""
import os

import numpy as np
import pytest

import oracle
from datagen import workloads as W
from tests.golden import make_golden
from tests.test_oracle_pins import _modular_closed_form

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _parse(name, aggs):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#"):
            continue
        f = line.split()
        key, count, rest = int(f[0]), int(f[1]), f[2:]
        sums, avgs = [], []
        for ag in aggs:
            sums.append(int(rest.pop(0)))
            avgs.append(float.fromhex(rest.pop(0)) if ag[0] == "avg" else None)
        rows.append((key, count, sums, avgs))
    return rows


@pytest.mark.parametrize("name", sorted(make_golden.CASES))
def test_oracle_reproduces_golden(name):
    wl = make_golden.CASES[name]()
    assert make_golden.render(wl) == open(os.path.join(GOLDEN, name)).read()


def test_modular_golden_matches_closed_form():
    wl = make_golden.CASES["modular_11550.txt"]()
    want = _modular_closed_form(11_550, 200)
    rows = _parse("modular_11550.txt", wl.query["aggs"])
    assert len(rows) == 150
    for key, count, sums, avgs in rows:
        cnt, s_qty, s_rev, s_disc = want[key]
        assert (count, sums[0], sums[1], sums[2], sums[3]) == (cnt, s_qty, s_rev, cnt, s_disc)


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(make_golden.CASES))
def test_cuda_path_reproduces_golden(name):
    from paper_2508_05029_gb300 import build
    from paper_2508_05029_gb300 import theseus as T
    build.build()
    wl = make_golden.CASES[name]()
    rows = _parse(name, wl.query["aggs"])
    with T.Engine(page_bytes=4 << 20, n_pages=32, batch_rows=8_192) as eng:
        for placement in (T.TP_DEVICE, T.TP_HOST_PAGES):
            ft = eng.table_from_numpy(wl.fact, placement=placement)
            dt = eng.table_from_numpy(wl.dim, placement=placement)
            p = eng.plan(ft, dt, wl.query)
            with p.execute() as r:
                assert r.n_groups == len(rows)
                assert np.array_equal(r.keys(), np.array([x[0] for x in rows], np.uint64))
                assert np.array_equal(r.counts(), np.array([x[1] for x in rows], np.int64))
                for a, ag in enumerate(wl.query["aggs"]):
                    if ag[0] == "count":
                        continue
                    w = r.sum_words(a)
                    got = [(int(hi) << 64 | int(lo)) - ((1 << 128) if int(hi) >> 63 else 0)
                           for lo, hi in w.astype(np.uint64)]
                    assert got == [x[2][a] for x in rows]
                    if ag[0] == "avg":
                        assert list(r.avg(a)) == [x[3][a] for x in rows]
            p.destroy()
            ft.destroy()
            dt.destroy()
