"""GPU tests of the serving loop (thr_server_*): with continuous batching,
every result equals the same query run alone (thr_query) and the CPU
oracle's, also with submissions and waits on different threads and with
single queries whose staging grows between cached graphs; requests that arrive while others run join later micro-batches;
micro-batches of several workers are in flight at once; the memory budget
bounds what is admitted; a budget smaller than one request still serves
every request, one at a time."""
import threading
import time

import numpy as np
import pytest

import oracle
import paper_1402_4466_gb300 as thr
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    return torch


@pytest.fixture(scope="module")
def served():
    """64 bitmaps over 2^20 + 77 rows with Zipf-like densities (odd i.i.d.,
    even clustered), as in the serving workload but smaller."""
    r = (1 << 20) + 77
    arrays = []
    for k in range(1, 65):
        p = min(0.3, 0.3 * k ** -1.1)
        arrays.append(synth.bernoulli(31, k, r, p) if k % 2 else synth.clustered(31, k, r, p))
    gw, goff = thr.encode_many(arrays, r)
    ostreams = [oracle.encode(w, r) for w in arrays]
    g = thr.idx_build_rle(gw, goff, r)
    return g, oracle.Index(ostreams, r), r


def _requests(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(3, 257))
        out.append((rng.integers(0, 64, n).astype(np.uint32), int(rng.integers(1, n + 1))))
    return out


def test_results_alone_and_in_the_mix(served):
    g, o, r = served
    reqs = _requests(1, 120)
    srv = thr.Server(g, workers=3, max_batch=16, mem_budget=1 << 30)
    try:
        tickets = [srv.submit(ids, T) for ids, T in reqs]  # a burst: they batch up
        got = [srv.wait(t) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    for (ids, T), (res, lat) in zip(reqs, got):
        alone = thr.thr_query(g, ids, T)
        assert np.array_equal(res, alone)
        assert lat > 0
    for (ids, T), (res, _) in zip(reqs[:30], got[:30]):
        assert np.array_equal(res, o.threshold(ids, T))
    assert st["done"] == len(reqs)
    assert st["batched_queries"] == len(reqs)
    assert st["batches"] < len(reqs)        # requests shared micro-batches
    assert st["max_batch"] > 1
    assert st["max_in_flight"] >= 2         # several micro-batches on the device at once


def test_arrivals_while_busy_join_later_batches(served):
    """A submitter thread keeps adding requests while earlier ones run; the
    waiter collects them in order.  Everything is served, in batches."""
    g, o, r = served
    reqs = _requests(2, 90)
    srv = thr.Server(g, workers=2, max_batch=8, mem_budget=1 << 30,
                     flags=thr.THR_POLICY_RULE)
    tickets = [None] * len(reqs)

    def submitter():
        for i, (ids, T) in enumerate(reqs):
            tickets[i] = srv.submit(ids, T)
            if i % 10 == 9:
                time.sleep(0.002)

    th = threading.Thread(target=submitter)
    th.start()
    results = []
    for i in range(len(reqs)):
        while tickets[i] is None:
            time.sleep(0.0005)
        results.append(srv.wait(tickets[i])[0])
    th.join()
    st = srv.stats()
    srv.close()
    for (ids, T), res in zip(reqs, results):
        assert np.array_equal(res, thr.thr_query(g, ids, T))
    assert st["done"] == len(reqs) and st["waiting"] == 0 and st["in_flight"] == 0


def test_memory_budget_bounds_admission(served):
    g, o, r = served
    reqs = _requests(3, 40)
    per_request = None
    # a budget below one request: one request at a time, all served
    srv = thr.Server(g, workers=3, max_batch=16, mem_budget=1)
    tickets = [srv.submit(ids, T) for ids, T in reqs]
    res = [srv.wait(t)[0] for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["max_in_flight"] == 1 and st["max_batch"] == 1 and st["batches"] == len(reqs)
    per_request = st["max_claimed_bytes"]
    for (ids, T), x in zip(reqs, res):
        assert np.array_equal(x, thr.thr_query(g, ids, T))
    # room for exactly three requests: never more than three claimed
    srv = thr.Server(g, workers=4, max_batch=16, mem_budget=3 * per_request)
    tickets = [srv.submit(ids, T) for ids, T in reqs]
    for t in tickets:
        srv.wait(t)
    st = srv.stats()
    srv.close()
    assert st["max_claimed_bytes"] <= 3 * per_request
    assert st["done"] == len(reqs)


def test_server_rejects_bad_requests(served):
    g, o, r = served
    srv = thr.Server(g, workers=1)
    try:
        with pytest.raises(thr.ThrError):
            srv.submit([0, 64], 1)  # id out of range
        with pytest.raises(thr.ThrError):
            srv.submit([], 1)
        with pytest.raises(thr.ThrError):
            srv.wait(12345)  # unknown ticket
        t = srv.submit([1, 2, 3], 2)
        small = np.zeros(1, np.uint64)
        res, _ = srv.wait(srv.submit([1, 2, 3], 2))
        assert np.array_equal(res, thr.thr_query(g, [1, 2, 3], 2))
        if len(res) > 1:
            with pytest.raises(thr.ThrError) as e:
                srv.wait(t, buf=small)
            assert e.value.status == thr.THR_E_NOSPACE
        else:
            srv.wait(t, buf=small)
    finally:
        srv.close()


def test_submit_while_waiting(served):
    """One thread submits while another waits, as a serving front end does:
    the table of live tickets grows (and rehashes) while waits are blocked
    on it.  Every result equals the same query run alone, and a sample the
    oracle's."""
    g, o, r = served
    rng = np.random.default_rng(37)
    reqs = []
    for _ in range(3000):
        n = int(rng.integers(2, 40))
        reqs.append((rng.integers(0, 64, n).astype(np.uint32), int(rng.integers(1, n + 1))))
    srv = thr.Server(g, workers=4, max_batch=16)
    tickets = [None] * len(reqs)
    got = [None] * len(reqs)

    def submitter():
        for i, (ids, T) in enumerate(reqs):
            tickets[i] = srv.submit(ids, T)
            if i % 50 == 0:
                time.sleep(0.0005)

    th = threading.Thread(target=submitter)
    th.start()
    try:
        for i in range(len(reqs)):
            while tickets[i] is None:
                time.sleep(0.0001)
            got[i] = srv.wait(tickets[i])[0]
    finally:
        th.join()
        srv.close()
    for i, (ids, T) in enumerate(reqs):
        assert np.array_equal(got[i], thr.thr_query(g, ids, T)), i
    for i in range(0, len(reqs), 60):
        ids, T = reqs[i]
        assert np.array_equal(got[i], o.threshold(ids, T)), i


def test_single_queries_while_staging_grows(served):
    """One thread, many single queries of varying size: the pinned staging
    a thread's calls share grows several times while graphs of earlier
    shapes are cached and later replayed (a new staging allocation can come
    back at the old address).  Every result equals the oracle's."""
    g, o, r = served
    for ids, T in _requests(1, 120):
        assert np.array_equal(thr.thr_query(g, ids, T), o.threshold(ids, T)), (len(ids), T)
