"""Request server: queries admitted continuously, batched as they arrive into
persistent launches (TP_SERVE_BATCH) or run on concurrent lanes; each result
equal to the oracle's and to the same query run alone."""
import threading
import time

import numpy as np
import pytest

import oracle
from datagen import workloads as W
from paper_2508_05029_gb300 import theseus as T
from tests.helpers import assert_matches_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2508_05029_gb300 import build
    build.build()
    eng = T.Engine(page_bytes=8 << 20, n_pages=256, batch_rows=1 << 20)
    # 4 shared dimensions, 16 requests with their own fact tables
    sz = W.config4_sizes(n_queries=16, fact_hi=4_000_000, dim_hi=300_000)
    wls = []
    for q in range(16):
        base = W.config4_query(q % 4, int(sz["fact"][q]), int(sz["dim"][q % 4]), int(sz["cutoff"][q]),
                               int(sz["groups"][q % 4]), fact_scale=0.01)
        fact = W.config4_query(q, int(sz["fact"][q]), int(sz["dim"][q % 4]), int(sz["cutoff"][q]),
                               int(sz["groups"][q % 4]), fact_scale=0.01).fact
        # fact keys drawn over this dimension's keys
        fact["fk"] = base.dim["pk"][np.arange(fact["fk"].size) * 7919 % base.dim["pk"].size]
        wls.append(W.Workload(f"req{q}", fact, base.dim, base.query))
    dims = [eng.table_from_numpy(wls[q].dim, placement=T.TP_DEVICE) for q in range(4)]
    facts = [eng.table_from_numpy(wl.fact, placement=T.TP_DEVICE) for wl in wls]
    plans = [eng.plan(facts[q], dims[q % 4], wls[q].query) for q in range(16)]
    refs = [oracle.run(wl) for wl in wls]
    yield eng, wls, plans, refs
    for p in plans:
        p.destroy()
    for t in facts + dims:
        t.destroy()
    eng.close()


def test_mix_matches_alone_and_oracle(setup):
    eng, wls, plans, refs = setup
    alone = []
    for p in plans:
        with p.execute() as r:
            alone.append((r.keys(), r.counts(), r.sum_words(1)))
    srv = T.Server(eng, workers=4, cache_dims=True)
    try:
        for rnd in range(2):
            tickets = [srv.submit(p) for p in plans]
            for q, t in enumerate(tickets):
                res, times = srv.wait(t, timeout_s=120)
                with res:
                    assert_matches_oracle(res, refs[q], wls[q].query["aggs"])
                    assert np.array_equal(res.sum_words(1), alone[q][2])
                assert times[0] <= times[1] <= times[2]
        st = srv.stats()
        assert st["completed"] == 32 and st["failed"] == 0
        assert st["cache_hits"] >= 28 and st["cache_misses"] == 4   # one build per dimension
        assert st["inflight_peak"] >= 2
    finally:
        srv.stop()


def _alone(plans):
    out = []
    for p in plans:
        with p.execute() as r:
            out.append((r.keys(), r.counts(), [r.sum_words(a) for a in (0, 1, 3)]))
    return out


def test_batched_mix_matches_alone_and_oracle(setup):
    eng, wls, plans, refs = setup
    alone = _alone(plans)
    srv = T.Server(eng, workers=2, batch=True)
    try:
        for rnd in range(3):
            tickets = [srv.submit(p) for p in (plans if rnd != 1 else plans[::-1])]
            order = list(range(16)) if rnd != 1 else list(range(15, -1, -1))
            for q, t in zip(order, tickets):
                res, times = srv.wait(t, timeout_s=120)
                with res:
                    assert_matches_oracle(res, refs[q], wls[q].query["aggs"])
                    assert np.array_equal(res.keys(), alone[q][0])
                    for a, w in zip((0, 1, 3), alone[q][2]):
                        assert np.array_equal(res.sum_words(a), w)
                assert times[0] <= times[1] <= times[2]
        st = srv.stats()
        assert st["completed"] == 48 and st["failed"] == 0
        assert 1 <= st["batches"] < 48          # requests shared launches
        assert st["inflight_peak"] >= 2
    finally:
        srv.stop()


def test_batched_requests_arriving_during_a_launch(setup):
    """Requests submitted from another thread in bursts, while earlier ones
    run, are admitted into later launches (a lone request on an idle GPU runs
    by itself); every result still equals its oracle."""
    eng, wls, plans, refs = setup
    srv = T.Server(eng, workers=1, batch=True)
    tickets = {}
    try:
        def submit_all():
            for k in range(64):
                q = (k * 7) % 16
                tickets[k] = (q, srv.submit(plans[q]))
                if k % 8 == 7:
                    time.sleep(0.002)
        th = threading.Thread(target=submit_all)
        th.start()
        th.join()
        for k in range(64):
            q, t = tickets[k]
            res, _ = srv.wait(t, timeout_s=120)
            with res:
                assert_matches_oracle(res, refs[q], wls[q].query["aggs"])
        st = srv.stats()
        assert st["completed"] == 64 and st["failed"] == 0 and st["batches"] >= 2
    finally:
        srv.stop()


def test_batched_and_lane_requests_mix(setup):
    """Plans a batched launch cannot take (a fact table in host pages) run on
    lanes beside the batches."""
    eng, wls, plans, refs = setup
    paged = [eng.table_from_numpy(wls[q].fact, placement=T.TP_HOST_PAGES) for q in range(3)]
    dims = [eng.table_from_numpy(wls[q].dim, placement=T.TP_DEVICE) for q in range(3)]
    pplans = [eng.plan(paged[q], dims[q], wls[q].query) for q in range(3)]
    srv = T.Server(eng, workers=2, batch=True)
    try:
        tickets = []
        for q in range(16):
            tickets.append((q, srv.submit(plans[q])))
            if q < 3:
                tickets.append((q, srv.submit(pplans[q])))
        for q, t in tickets:
            res, _ = srv.wait(t, timeout_s=120)
            with res:
                assert_matches_oracle(res, refs[q], wls[q].query["aggs"])
        st = srv.stats()
        assert st["completed"] == 19 and st["failed"] == 0 and st["batches"] >= 1
    finally:
        srv.stop()
        for p in pplans:
            p.destroy()
        for t in paged + dims:
            t.destroy()


def test_second_waiter_on_a_ticket_is_refused(setup):
    """While one thread waits on a ticket, a second tp_wait on it returns
    TP_E_INVALID instead of sharing (and later freeing) the request."""
    eng, wls, plans, refs = setup
    big = max(range(16), key=lambda q: wls[q].n_fact)
    srv = T.Server(eng, workers=1, cache_dims=False)   # one lane: the requests run one by one
    try:
        ahead = [srv.submit(plans[big]) for _ in range(40)]
        last = ahead[-1]
        got = {}

        def first():
            got["r"] = srv.wait(last, timeout_s=120)
        th = threading.Thread(target=first)
        th.start()
        seen = set()
        lib = eng.lib
        import ctypes
        while th.is_alive() and "invalid" not in seen:
            r = ctypes.c_void_p()
            code = lib.tp_wait(srv.h, last, 0, ctypes.byref(r), None)
            seen.add(T.STATUS_NAMES[code])
            assert code in (T.TP_E_INVALID, T.TP_E_TIMEOUT)
            time.sleep(0.0002)
        th.join()
        res, _ = got["r"]
        with res:
            assert_matches_oracle(res, refs[big], wls[big].query["aggs"])
        for t in ahead[:-1]:
            srv.wait(t, timeout_s=120)[0].free()
        assert "invalid" in seen
    finally:
        srv.stop()


@pytest.mark.parametrize("batch,workers", [(False, 4), (False, 2), (True, 2)])
def test_budget_admission_defers_not_fails(setup, batch, workers):
    eng, wls, plans, refs = setup
    used, cap = eng.budget()
    # room for roughly one request at a time beyond the placed tables
    eng.set_budget(used + (48 << 20))
    srv = T.Server(eng, workers=workers, cache_dims=False, batch=batch)
    try:
        tickets = [srv.submit(p) for p in plans]
        for q, t in enumerate(tickets):
            res, _ = srv.wait(t, timeout_s=120)
            with res:
                assert_matches_oracle(res, refs[q], wls[q].query["aggs"])
        st = srv.stats()
        assert st["failed"] == 0
    finally:
        srv.stop()
        eng.set_budget(cap)


@pytest.mark.parametrize("batch", [False, True])
def test_request_that_cannot_fit_fails_alone(setup, batch):
    eng, wls, plans, refs = setup
    used, cap = eng.budget()
    eng.set_budget(used + 1024)
    srv = T.Server(eng, workers=2, cache_dims=False, batch=batch)
    try:
        t = srv.submit(plans[0])
        with pytest.raises(T.TPError) as e:
            srv.wait(t, timeout_s=60)
        assert e.value.status == "budget"
    finally:
        srv.stop()
        eng.set_budget(cap)


@pytest.mark.parametrize("batch", [False, True])
def test_errors_stay_with_their_request(setup, batch):
    eng, wls, plans, refs = setup
    bad = {k: v.copy() for k, v in wls[0].dim.items()}
    bad["pk"][1] = bad["pk"][2]
    dbad = eng.table_from_numpy(bad, placement=T.TP_DEVICE)
    fbad = eng.table_from_numpy(wls[0].fact, placement=T.TP_DEVICE)
    pbad = eng.plan(fbad, dbad, wls[0].query)
    srv = T.Server(eng, workers=3, cache_dims=True, batch=batch)
    try:
        tickets = [srv.submit(plans[1]), srv.submit(pbad), srv.submit(plans[2])]
        res, _ = srv.wait(tickets[0], timeout_s=60)
        with res:
            assert_matches_oracle(res, refs[1], wls[1].query["aggs"])
        with pytest.raises(T.TPError) as e:
            srv.wait(tickets[1], timeout_s=60)
        assert e.value.status == "dup_key"
        res, _ = srv.wait(tickets[2], timeout_s=60)
        with res:
            assert_matches_oracle(res, refs[2], wls[2].query["aggs"])
    finally:
        srv.stop()
        pbad.destroy()
        dbad.destroy()
        fbad.destroy()
