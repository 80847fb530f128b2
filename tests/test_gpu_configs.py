"""GPU parity at the shapes of the batched-similarity and serving workloads,
against the CPU oracle (the plain definition of Sec. 2: the rows counted in at
least T of the query's inputs), word for word.

* similarity shape: r = 2^24 rows, queries of N ~ U[10, 200] Zipf-drawn terms
  with a planted prototype row and T = ceil(N / 2), 256 of them in one
  thr_query_batch call under the learned policy (the shipped cost model),
  with the launch configuration from the autotuner and the queries cut into
  several chunks.  The term count is reduced from 2^16 to 2048 (densities
  min(0.3, C k^-1.1) rescaled to sum to 110 * 2048 / 2^16) so that the index
  and the oracle's work fit a test.
* serving shape: r = 2^26 rows, 384 bitmaps with densities 0.3 k^-1.1 (odd k
  i.i.d., even k clustered), requests of N ~ U[3, 256] ids drawn with
  replacement and T ~ U[1, N] through thr_server_* with several workers
  under the learned policy.

The oracle runs row-partitioned over the host cores (the partitioned
ScanCount is pinned against brute force in tests/oracle_pins.py).
"""
import os

import numpy as np
import pytest

import oracle
import paper_1402_4466_gb300 as thr
import synth
from paper_1402_4466_gb300 import selector_weights, workloads

pytestmark = pytest.mark.gpu

POOL = min(16, os.cpu_count() or 1)


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    return torch


def _oracle_index(words, offsets, r):
    streams = [words[int(offsets[i]): int(offsets[i + 1])] for i in range(len(offsets) - 1)]
    return oracle.Index(streams, r)


def test_similarity_shape_batch_learned_policy(cuda):
    torch = cuda
    nb, r, nq = 2048, 1 << 24, 256
    dens = synth.similarity_densities(nb, mean_len=110.0 * nb / (1 << 16))
    queries, planted, protos = synth.similarity_queries(3, nq, dens, r)
    jobs = [(3, k, r, float(dens[k]), False, planted.get(k)) for k in range(nb)]
    words, offsets = workloads.encode_family(jobs, POOL)
    idx = thr.idx_build_rle(words, offsets, r)
    sel = selector_weights.attach(idx)
    o = _oracle_index(words, offsets, r)
    cores = oracle.load().max_threads()
    try:
        thr.thr_autotune(idx, queries[:64], flags=thr.THR_POLICY_LEARNED, reps=2)
        pool = torch.empty(nq * (idx.nwords + 1), dtype=torch.int64, device="cuda")
        os.environ["THR_MAX_SLOTS"] = "96"  # three chunks
        try:
            off, ln, _ = thr.thr_query_batch(idx, queries, pool=pool,
                                             flags=thr.THR_POLICY_LEARNED)
            info = thr.thr_last_batch_info()
        finally:
            del os.environ["THR_MAX_SLOTS"]
        assert info["chunks"] >= 2
        host = pool.cpu().numpy().view(np.uint64)
        for k, (ids, T) in enumerate(queries):
            want = o.threshold_parts(ids, T, cores)
            got = host[int(off[k]): int(off[k] + ln[k])]
            assert np.array_equal(got, want), f"query {k}: n={len(ids)} T={T}"
        # the same call again relaunches the cached graph: same results
        off2, ln2, _ = thr.thr_query_batch(idx, queries, pool=pool,
                                           flags=thr.THR_POLICY_LEARNED)
        host2 = pool.cpu().numpy().view(np.uint64)
        for k in range(0, nq, 17):
            assert np.array_equal(host2[int(off2[k]): int(off2[k] + ln2[k])],
                                  host[int(off[k]): int(off[k] + ln[k])])
    finally:
        thr.set_selector(idx, None)
        del sel
        idx.close()


def test_serving_shape_server_learned_policy():
    nb, r = 384, 1 << 26
    dens = synth.serving_densities(nb)
    jobs = [(5, k, r, float(dens[k - 1]), k % 2 == 0, None) for k in range(1, nb + 1)]
    words, offsets = workloads.encode_family(jobs, POOL)
    idx = thr.idx_build_rle(words, offsets, r)
    sel = selector_weights.attach(idx)
    o = _oracle_index(words, offsets, r)
    cores = oracle.load().max_threads()
    rng = np.random.default_rng(5)
    reqs = []
    for _ in range(40):
        n = int(rng.integers(3, 257))
        reqs.append((rng.integers(0, nb, n).astype(np.uint32), int(rng.integers(1, n + 1))))
    srv = thr.Server(idx, workers=4, max_batch=8, mem_budget=2 << 30,
                     flags=thr.THR_POLICY_LEARNED)
    try:
        tickets = [srv.submit(ids, T) for ids, T in reqs]
        got = [srv.wait(t) for t in tickets]
    finally:
        srv.close()
    try:
        for k, ((ids, T), (res, _lat)) in enumerate(zip(reqs, got)):
            want = o.threshold_parts(ids, T, cores)
            assert np.array_equal(res, want), f"request {k}: n={len(ids)} T={T}"
    finally:
        thr.set_selector(idx, None)
        del sel
        idx.close()
