"""GPU parity of row-sharded execution and of very large queries (the two
questions of Sec. 9: partitioning the problem, and N = 10^6 inputs), against
the CPU oracle, word for word.

* Shards: the 64 x 2^26 many-criteria bitmaps cut into G = 2, 3, 5 row
  ranges (64-row aligned), one index per shard on this GPU (thr_rle_slice),
  each shard queried with thr_query and the results stitched
  (thr_rle_stitch): equal to the oracle's result over all rows, at the
  benchmark's thresholds and at random ids and thresholds.
* Opt-threshold over shards: each shard's profiling pass (its answer and
  count histogram, thr_query_opt_hist), the histograms combined
  (sharded.combine_opt), then the threshold query on every shard: equal to
  the oracle's opt-threshold answer and result over all rows.
* A million inputs: n = 10^6 ids drawn with repetition from 48 bitmaps
  (20-bit counters), thresholds from 1 to n + 1, single queries and a batch,
  against the per-row count over the uncompressed bits (the definition of
  Sec. 2) and, for two thresholds, the oracle.
"""
import numpy as np
import pytest

import oracle
import paper_1402_4466_gb300 as thr
import synth
from paper_1402_4466_gb300 import sharded

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    return torch


@pytest.fixture(scope="module")
def many(many_criteria_full):
    arrays, r = many_criteria_full
    words, offsets = thr.encode_many(arrays, r)
    o = oracle.Index([words[int(offsets[i]):int(offsets[i + 1])]
                      for i in range(len(offsets) - 1)], r)
    return words, offsets, r, o


def test_row_shards_stitched_equal_the_whole(many):
    words, offsets, r, o = many
    cores = oracle.load().max_threads()
    rng = np.random.default_rng(41)
    queries = [(list(range(synth.MANY_N)), T) for T in synth.MANY_TS]
    for _ in range(3):
        n = int(rng.integers(2, 100))
        queries.append((rng.integers(0, synth.MANY_N, n).tolist(), int(rng.integers(1, n + 1))))
    want = [o.threshold_parts(ids, T, cores) for ids, T in queries]
    for G in (2, 3, 5):
        ss = sharded.ShardSet(words, offsets, r, G)
        try:
            for (ids, T), w in zip(queries, want):
                assert np.array_equal(ss.query(ids, T), w), (G, len(ids), T)
        finally:
            ss.close()


def test_opt_threshold_over_row_shards(many):
    words, offsets, r, o = many
    ids = list(range(synth.MANY_N))
    ss = sharded.ShardSet(words, offsets, r, 3)
    try:
        for K in (1, 1000):
            T, got = ss.query_opt(ids, K)
            Tw, want = o.opt_threshold(ids, K)
            assert T == Tw
            assert np.array_equal(got, want)
    finally:
        ss.close()


def test_million_inputs():
    r = 640 + 17
    arrays = [synth.bernoulli(43, k, r, p) for k, p in enumerate(np.linspace(0.005, 0.1, 40))]
    arrays += [synth.clustered(43, 100 + k, r, 0.1) for k in range(8)]
    gw, goff = thr.encode_many(arrays, r)
    g = thr.idx_build_rle(gw, goff, r)
    o = oracle.Index([oracle.encode(a, r) for a in arrays], r)
    rng = np.random.default_rng(43)
    n = 1_000_000
    ids = rng.integers(0, len(arrays), n).astype(np.uint32)
    bits = np.stack([synth.words_to_bits(a, r) for a in arrays]).astype(np.int64)

    def definition(q, T):  # Sec. 2: rows counted at least T times over the multiset q
        mult = np.bincount(q, minlength=len(arrays))
        return oracle.encode(synth.rows_to_words(np.nonzero(mult @ bits >= T)[0], r), r)

    try:
        for T in (1, 2, 25_000, 100_000, 150_000, 180_000, n // 2, n + 1):
            want = definition(ids, T)
            assert np.array_equal(thr.thr_query(g, ids, T), want), T
            if T in (25_000, 150_000):
                assert np.array_equal(o.threshold(ids, T), want)
        qs = [(ids, 150_000), (ids[: n // 2], 60_000), (ids[:1000], 100)]
        off, ln, pool = thr.thr_query_batch(g, qs, flags=thr.THR_NO_SHARE)
        for k, (q, T) in enumerate(qs):
            assert np.array_equal(pool[int(off[k]): int(off[k] + ln[k])], definition(q, T))
    finally:
        g.close()
