"""Serving loop: requests with their own k and recall target, submitted from
several threads while others are on the GPU, return exactly what the same
queries return alone (leafi_search_mixed), and admission respects the budget."""
import threading

import numpy as np
import pytest

import fixtures as fx
import paper_2502_01836_b300 as lf
from paper_2502_01836_b300.workflow import enhance

pytestmark = pytest.mark.gpu

M = 128
KMAX = 20


@pytest.fixture(scope="module")
def served():
    X = fx.random_walk(30000, M, seed=81)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=800, wave=8, device=0))
    enhance(idx, 12, kclasses=(1, 10, 20), max_epochs=40, patience=4)
    yield X, idx
    lf.leafi_free(idx)


def _alone(idx, Q, k, t):
    ids = np.zeros((len(Q), KMAX), np.int64)
    d = np.zeros((len(Q), KMAX), np.float32)
    lf.leafi_search_mixed(idx, Q, k, t, KMAX, ids, d)
    return ids, d


@pytest.mark.parametrize("max_batch", [256, 700])
def test_results_alone_equal_results_in_the_mix(served, max_batch):
    X, idx = served
    rng = np.random.default_rng(82)
    reqs = []
    for r in range(16):
        nq = int(rng.integers(1, 90))
        Q = fx.test_queries(X, nq, seed=1000 + r)
        k = rng.choice([1, 5, 10, 20], nq).astype(np.int32)
        t = rng.choice([0.9, 0.95, 0.99, 1.0], nq).astype(np.float64)
        reqs.append((Q, k, t))
    sv = lf.leafi_serve_start(idx, kmax=KMAX, max_batch=max_batch, max_wait_ms=0.5)
    try:
        tickets = [None] * len(reqs)

        def submit(lo, hi):
            for r in range(lo, hi):
                tickets[r] = lf.leafi_serve_submit(sv, *reqs[r])

        th = [threading.Thread(target=submit, args=(4 * i, 4 * i + 4)) for i in range(4)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        for r, (Q, k, t) in enumerate(reqs):
            ids = np.zeros((len(Q), KMAX), np.int64)
            d = np.zeros((len(Q), KMAX), np.float32)
            done, lat = False, 0.0
            for _ in range(200):
                done, lat = lf.leafi_serve_poll(sv, tickets[r], ids, d, wait_ms=50.0)
                if done:
                    break
            assert done and lat > 0.0
            a_ids, a_d = _alone(idx, Q, k, t)
            assert np.array_equal(ids, a_ids) and np.array_equal(d, a_d), r
        st = lf.leafi_serve_get_stats(sv)
        assert st["requests"] == len(reqs)
        assert st["queries"] == sum(len(q) for q, _, _ in reqs)
        assert 1 <= st["batches"] <= st["queries"]
    finally:
        lf.leafi_serve_stop(sv)


def test_admission_budget(served):
    X, idx = served
    Q = fx.test_queries(X, 50, seed=83)
    k = np.full(50, 5, np.int32)
    t = np.full(50, 1.0)
    per_query = M * 4 + 4 + 8 + KMAX * 12
    sv = lf.leafi_serve_start(idx, kmax=KMAX, max_bytes=60 * per_query)
    try:
        t1 = lf.leafi_serve_submit(sv, Q, k, t)
        with pytest.raises(lf.LeafiError) as e:
            lf.leafi_serve_submit(sv, Q, k, t)
        assert e.value.status == lf.EAGAIN
        ids = np.zeros((50, KMAX), np.int64)
        d = np.zeros((50, KMAX), np.float32)
        done = False
        for _ in range(200):
            done, _ = lf.leafi_serve_poll(sv, t1, ids, d, wait_ms=50.0)
            if done:
                break
        assert done
        t2 = lf.leafi_serve_submit(sv, Q, k, t)   # the budget was released by the poll
        for _ in range(200):
            done, _ = lf.leafi_serve_poll(sv, t2, ids, d, wait_ms=50.0)
            if done:
                break
        assert done
        a_ids, a_d = _alone(idx, Q, k, t)
        assert np.array_equal(ids, a_ids) and np.array_equal(d, a_d)
    finally:
        lf.leafi_serve_stop(sv)


def test_requests_admitted_while_batches_are_in_flight(served):
    """Continuous batching: requests submitted while earlier batches are on the
    GPU are admitted (counted by the server) and join later batches; their
    results equal what the same queries return alone."""
    X, idx = served
    big = fx.test_queries(X, 2000, seed=84)              # eight batches of 256
    kb = np.full(2000, 10, np.int32)
    tb = np.full(2000, 0.95)
    small = [fx.test_queries(X, 5, seed=85 + i) for i in range(20)]
    ks = [np.full(5, 1 + i % KMAX, np.int32) for i in range(20)]
    ts = [np.full(5, (0.9, 0.99, 1.0)[i % 3]) for i in range(20)]
    sv = lf.leafi_serve_start(idx, kmax=KMAX, max_batch=256, max_wait_ms=0.2)
    try:
        tb_ticket = lf.leafi_serve_submit(sv, big, kb, tb)
        tickets = [lf.leafi_serve_submit(sv, small[i], ks[i], ts[i]) for i in range(20)]
        st = None

        def collect(ticket, nq):
            ids = np.zeros((nq, KMAX), np.int64)
            d = np.zeros((nq, KMAX), np.float32)
            for _ in range(400):
                done, _ = lf.leafi_serve_poll(sv, ticket, ids, d, wait_ms=50.0)
                if done:
                    return ids, d
            raise AssertionError("request did not finish")

        got = [collect(t, 5) for t in tickets]
        gb = collect(tb_ticket, 2000)
        st = lf.leafi_serve_get_stats(sv)
        assert st["admitted_in_flight"] >= 1
        assert st["device_bytes"] > 0
        for i in range(20):
            a_ids, a_d = _alone(idx, small[i], ks[i], ts[i])
            assert np.array_equal(got[i][0], a_ids) and np.array_equal(got[i][1], a_d), i
        a_ids, a_d = _alone(idx, big[:300], kb[:300], tb[:300])
        assert np.array_equal(gb[0][:300], a_ids) and np.array_equal(gb[1][:300], a_d)
    finally:
        lf.leafi_serve_stop(sv)
