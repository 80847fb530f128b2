"""GPU parity of opt-threshold queries (thr_query_opt / thr_query_opt_batch,
through the C ABI): the answer T and its result stream equal the CPU
oracle's exactly, for K = 1 (the largest count) and larger K, on tiny random
cases, several-tile cases with ragged tails and more inputs than one chunk,
wide counters (n > 255), similarity queries with a planted best match, the
64 x 2^26 many-criteria workload at full size, and the degenerate cases
(every row counted 0, K > r, K = r, a single full bitmap)."""
import numpy as np
import pytest

import oracle
import oracle_pins
import paper_1402_4466_gb300 as thr
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    return torch


class Pair:
    def __init__(self, word_arrays, r):
        self.r = r
        gw, goff = thr.encode_many(word_arrays, r)
        ostreams = [oracle.encode(w, r) for w in word_arrays]
        self.g = thr.idx_build_rle(gw, goff, r)
        self.o = oracle.Index(ostreams, r)

    def check(self, ids, K):
        T, got = thr.thr_query_opt(self.g, ids, K)
        Tw, want = self.o.opt_threshold(ids, K)
        assert T == Tw, f"n={len(ids)} K={K} r={self.r}: T {T} vs {Tw}"
        assert np.array_equal(got, want), f"n={len(ids)} K={K} r={self.r}: result differs"
        return T


def from_ints(bitsets, r):
    return Pair([oracle_pins.int_to_words(b, r) for b in bitsets], r)


def test_tiny_random_every_k():
    rng = np.random.default_rng(303)
    for _ in range(15):
        n = int(rng.integers(1, 9))
        r = int(rng.choice([1, 63, 64, 65, 1000, 9000, 40000]))
        p = from_ints(oracle_pins.random_bitsets(rng, n, r), r)
        ids = rng.integers(0, n, int(rng.integers(1, 2 * n + 1))).tolist()
        for K in sorted({1, 2, 3, 7, 64, max(1, r // 2), r, r + 1}):
            p.check(ids, K)


def test_several_tiles_chunks_and_wide_counters():
    r = (1 << 18) + 77
    words, _ = synth.many_criteria(21, 30, r)
    p = Pair(words, r)
    for K in (1, 2, 10, 100, 5000, r // 3, r):
        p.check(list(range(30)), K)
    rng = np.random.default_rng(22)
    ids = rng.integers(0, 30, size=300).tolist()  # n > 128 (chunks), 2^9 > n: 9-bit counts
    for K in (1, 50, 20_000):
        p.check(ids, K)
    ids = rng.integers(0, 30, size=1100).tolist()  # 11-bit counts
    for K in (1, 3000):
        p.check(ids, K)


def test_similarity_planted_match():
    r = 1 << 17
    words = []
    rng = np.random.default_rng(9)
    for i in range(40):
        words.append(synth.bernoulli(9, i, r, float(10 ** rng.uniform(-3, -0.7))))
    # rows 777 and 90_000 are in 35 and 33 of the first 36 inputs
    for i in range(36):
        w = words[i]
        if i < 35:
            w[777 // 64] |= np.uint64(1) << np.uint64(777 % 64)
        if i < 33:
            w[90_000 // 64] |= np.uint64(1) << np.uint64(90_000 % 64)
    p = Pair(words, r)
    ids = list(range(36))
    assert p.check(ids, 1) >= 35
    assert p.check(ids, 2) >= 33
    for K in (3, 10, 1000):
        p.check(ids, K)


def test_degenerate_cases():
    r = 5000
    p = Pair([np.zeros(synth.nwords(r), np.uint64)] * 2, r)
    assert p.check([0, 1], 1) == 0       # every row counts 0: T = 0, every row
    full = oracle_pins.int_to_words((1 << r) - 1, r)
    p = Pair([full, np.zeros(synth.nwords(r), np.uint64)], r)
    assert p.check([0, 0, 0, 1], 1) == 3
    assert p.check([0, 0, 0, 1], r) == 3
    assert p.check([0, 0, 0, 1], r + 1) == 0
    p = from_ints([1, 1 << 63, (1 << 64) | 1], 65)
    assert p.check([0, 1, 2], 1) == 2
    p.check([2, 2, 0], 1)
    with pytest.raises(thr.ThrError):
        thr.thr_query_opt(p.g, [0], 0)


def test_batch_equals_single_queries():
    r = (1 << 19) + 5
    words, _ = synth.many_criteria(31, 24, r)
    p = Pair(words, r)
    rng = np.random.default_rng(32)
    queries = []
    for i in range(12):
        n = int(rng.integers(2, 60))
        ids = rng.integers(0, 24, n).tolist()
        K = int(rng.choice([1, 1, 4, 100, 10_000]))
        queries.append((ids, K))
    T, off, ln, pool = thr.thr_query_opt_batch(p.g, queries)
    for q, (ids, K) in enumerate(queries):
        Tw, want = p.o.opt_threshold(ids, K)
        assert int(T[q]) == Tw, (q, K)
        got = pool[int(off[q]): int(off[q]) + int(ln[q])]
        assert np.array_equal(got, want), q


def test_many_criteria_full_size(many_criteria_full):
    words, r = many_criteria_full
    p = Pair(words, r)
    ids = list(range(synth.MANY_N))
    for K in (1, 1000):
        p.check(ids, K)
