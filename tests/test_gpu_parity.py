"""GPU parity: every result of the CUDA library, called through its C ABI,
equals the CPU oracle's word for word (exact integer/bitwise arithmetic, so
the tolerance is zero).  Inputs are seeded synthetic bitmaps; each side
encodes them with its own codec and the two encodings must agree.

Sizes: tiny random cases (all T), several-tile cases with ragged tails, the
8 x 2^20 plain workload, the 64 x 2^26 many-criteria workload at full size in
the launch configuration the benchmark times, and edge cases (r = 1, ragged
last words, empty and full bitmaps, duplicated ids, T = 0, T > N, more
inputs than one chunk, undersized outputs)."""
import numpy as np
import pytest

import oracle
import oracle_pins
import paper_1402_4466_gb300 as thr
import synth
from golden import bits_row0_first, hex_words, read_kv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    return torch


class Pair:
    """The same bitmaps as a GPU index and an oracle index."""

    def __init__(self, word_arrays, r):
        self.r = r
        gw, goff = thr.encode_many(word_arrays, r)
        ostreams = [oracle.encode(w, r) for w in word_arrays]
        ow, ooff = oracle.concat(ostreams)
        assert np.array_equal(gw, ow) and np.array_equal(goff, ooff), \
            "library and oracle encoders disagree"
        self.g = thr.idx_build_rle(gw, goff, r)
        self.o = oracle.Index(ostreams, r)

    def check(self, ids, T, flags=0):
        got = thr.thr_query(self.g, ids, T, flags=flags)
        want = self.o.threshold(ids, T)
        if not np.array_equal(got, want):
            gr = oracle.decode(got, self.r) if oracle.validate(got, self.r) == 0 else None
            wr = oracle.decode(want, self.r)
            msg = f"T={T} n={len(ids)} r={self.r}: lengths {len(got)} vs {len(want)}"
            if gr is None:
                msg += "; GPU stream is not canonical"
            else:
                d = np.setxor1d(gr, wr)
                msg += f"; {len(d)} rows differ, first {d[:8].tolist()}"
            pytest.fail(msg)
        return got


def from_ints(bitsets, r):
    return Pair([oracle_pins.int_to_words(b, r) for b in bitsets], r)


def test_paper_examples():
    g = read_kv("fig1_threshold.txt")
    p = from_ints([bits_row0_first(g[k]) for k in ("B1", "B2", "B3")], int(g["r"]))
    for T in range(0, 5):
        p.check([0, 1, 2], T)
    g = read_kv("rbmrg_ewah.txt")
    B = [oracle_pins.words_to_int(hex_words(g[k])) for k in ("B1", "B2", "B3", "B4")]
    p = from_ints(B, int(g["r"]))
    got = p.check([0, 1, 2, 3], 3)
    assert oracle.decode(got, p.r).tolist() == oracle_pins.rows_of(
        oracle_pins.words_to_int(hex_words(g["result"])))
    for T in range(0, 6):
        p.check([0, 1, 2, 3], T)


def test_random_tiny_all_thresholds():
    rng = np.random.default_rng(101)
    for _ in range(30):
        n = int(rng.integers(1, 13))
        r = int(rng.choice([1, 5, 63, 64, 65, 200, 1000, 4096, 8191, 9000, 40000]))
        p = from_ints(oracle_pins.random_bitsets(rng, n, r), r)
        for T in range(0, n + 2):
            p.check(list(range(n)), T)
        ids = rng.integers(0, n, size=int(rng.integers(1, 20))).tolist()
        for T in (0, 1, 2, len(ids) // 2, len(ids), len(ids) + 1):
            p.check(ids, T)


@pytest.mark.parametrize("r", [(1 << 18) + 37, 9 * 512 * 64, 3 * 512 * 64 + 64 * 5 + 1])
def test_several_tiles_ragged(r):
    words, _ = synth.many_criteria(11, 24, r)
    p = Pair(words, r)
    for T in list(range(0, 8)) + [11, 12, 13, 20, 23, 24, 25]:
        p.check(list(range(24)), T)


def test_plain_workload():
    r = synth.PLAIN_R
    p = Pair(synth.plain(0, synth.PLAIN_N, r, synth.PLAIN_P), r)
    for T in range(0, synth.PLAIN_N + 2):
        p.check(list(range(synth.PLAIN_N)), T)


def test_many_criteria_full_size(many_criteria_full):
    """64 bitmaps over 2^26 rows; the thresholds the benchmark times."""
    words, r = many_criteria_full
    p = Pair(words, r)
    ids = list(range(synth.MANY_N))
    for T in synth.MANY_TS:
        p.check(ids, T)
    p.check(ids, 1)
    p.check(ids, 64)


def test_more_inputs_than_one_chunk():
    r = 50_000
    words, _ = synth.many_criteria(5, 40, r)
    p = Pair(words, r)
    rng = np.random.default_rng(5)
    ids = rng.integers(0, 40, size=600).tolist()
    for T in (0, 1, 2, 30, 150, 300, 450, 599, 600, 601):
        p.check(ids, T)


def test_edge_bitmaps():
    for r in (1, 2, 63, 64, 65, 128 * 64, 128 * 64 + 1, 512 * 64, 512 * 64 + 63):
        full = (1 << r) - 1
        alt = int("01" * ((r + 1) // 2), 2) & full
        B = [0, full, 1 << (r - 1), full ^ 1, alt]
        p = from_ints(B, r)
        for T in range(0, 7):
            p.check([0, 1, 2, 3, 4], T)
        p.check([1], 1)
        p.check([0], 1)
        p.check([1, 1, 1], 3)


def test_duplicate_ids_and_single_input():
    r = 70_000
    words, _ = synth.many_criteria(9, 6, r)
    p = Pair(words, r)
    for T in range(0, 5):
        p.check([2, 2, 2], T)
        p.check([4], T)
        p.check([0, 1, 1, 3, 3, 3], T)


def test_device_output_and_nospace(cuda):
    torch = cuda
    r = (1 << 16) + 11
    words, _ = synth.many_criteria(3, 10, r)
    p = Pair(words, r)
    ids = list(range(10))
    want = p.o.threshold(ids, 3)
    out = torch.zeros(len(want) + 5, dtype=torch.int64, device="cuda")
    n = thr.thr_query(p.g, ids, 3, out=out)
    assert n == len(want)
    assert np.array_equal(out[:n].cpu().numpy().view(np.uint64), want)
    small = torch.zeros(len(want) - 1, dtype=torch.int64, device="cuda")
    with pytest.raises(thr.ThrError) as e:
        thr.thr_query(p.g, ids, 3, out=small)
    assert e.value.status == thr.THR_E_NOSPACE
    st, need = thr.thr_query_raw(p.g, ids, 3, small.data_ptr(), small.numel(),
                                 thr.THR_OUT_DEVICE)
    assert st == thr.THR_E_NOSPACE and need == len(want)
    host = np.zeros(len(want) - 1, dtype=np.uint64)
    st, need = thr.thr_query_raw(p.g, ids, 3, host.ctypes.data, host.size, 0)
    assert st == thr.THR_E_NOSPACE and need == len(want)


def test_batch_matches_single_queries(cuda):
    r = 100_000
    words, _ = synth.many_criteria(4, 16, r)
    p = Pair(words, r)
    rng = np.random.default_rng(4)
    queries = []
    for _ in range(12):
        n = int(rng.integers(1, 30))
        ids = rng.integers(0, 16, size=n).tolist()
        queries.append((ids, int(rng.integers(0, n + 2))))
    off, ln, pool = thr.thr_query_batch(p.g, queries)
    for q, (ids, T) in enumerate(queries):
        got = pool[int(off[q]): int(off[q]) + int(ln[q])]
        assert np.array_equal(got, p.o.threshold(ids, T))


def test_invalid_arguments():
    p = from_ints([5, 7], 64)
    with pytest.raises(thr.ThrError) as e:
        thr.thr_query(p.g, [0, 2], 1)
    assert e.value.status == thr.THR_E_INVAL
    with pytest.raises(thr.ThrError) as e:
        thr.thr_query(p.g, [], 1)
    assert e.value.status == thr.THR_E_INVAL


# ---- the ScanCount counting kernel (per-row byte counters, Sec. 5.1)

SC = thr.THR_VARIANT_SCANCOUNT


def test_scancount_random_tiny_all_thresholds():
    rng = np.random.default_rng(202)
    for _ in range(20):
        n = int(rng.integers(1, 13))
        r = int(rng.choice([1, 63, 64, 65, 1000, 4096, 9000, 40000]))
        p = from_ints(oracle_pins.random_bitsets(rng, n, r), r)
        for T in range(0, n + 2):
            p.check(list(range(n)), T, SC)


def test_scancount_several_tiles_and_duplicates():
    r = (1 << 18) + 37
    words, _ = synth.many_criteria(12, 24, r)
    p = Pair(words, r)
    for T in (1, 2, 3, 5, 12, 24, 25):
        p.check(list(range(24)), T, SC)
    rng = np.random.default_rng(12)
    ids = rng.integers(0, 24, size=200).tolist()  # two chunks, n <= 255
    for T in (1, 2, 10, 50, 100, 200):
        p.check(ids, T, SC)
    ids = rng.integers(0, 24, size=300).tolist()  # n > 255: 16-bit counters
    for T in (1, 30, 256, 300):
        p.check(ids, T, SC)
    ids = rng.integers(0, 24, size=1200).tolist()  # four record chunks, 16-bit counters
    for T in (2, 60, 700):
        p.check(ids, T, SC)


def test_scancount_wide_counters_sparse_and_fallback():
    """Very sparse bitmaps (the case ScanCount is for) with more than 255
    inputs: counts past 255 in 16-bit counters, ones fills counted per word;
    above 65535 inputs the carry-save kernel runs instead."""
    r = (1 << 17) + 9
    arrays = [synth.bernoulli(33, k, r, 1e-3) for k in range(30)]
    arrays.append(synth.rows_to_words(np.arange(1000, 9000), r))  # ones fills
    p = Pair(arrays, r)
    rng = np.random.default_rng(33)
    ids = rng.integers(0, 31, size=2000).tolist() + [30] * 300
    for T in (1, 2, 3, 250, 256, 300, 2300):
        p.check(ids, T, SC)
    big = rng.integers(0, 31, size=70_000).tolist()
    for T in (2, 3000):
        p.check(big, T, SC)


def test_scancount_many_criteria_full_size(many_criteria_full):
    words, r = many_criteria_full
    p = Pair(words, r)
    for T in (2, 16):
        p.check(list(range(synth.MANY_N)), T, SC)


# ---- carry-save counters with the position-major decode of mixed inputs

POS = thr.THR_VARIANT_POSITION


def test_position_random_tiny_all_thresholds():
    rng = np.random.default_rng(303)
    for _ in range(20):
        n = int(rng.integers(1, 13))
        r = int(rng.choice([1, 63, 64, 65, 1000, 4096, 9000, 40000]))
        p = from_ints(oracle_pins.random_bitsets(rng, n, r), r)
        for T in range(0, n + 2):
            p.check(list(range(n)), T, POS)


def test_position_clustered_runs_and_chunks():
    """Clustered bitmaps put ones-fill words inside mixed subtiles; more
    than 32 mixed inputs per subtile take several transposed batches, more
    than 128 inputs several record chunks."""
    r = (1 << 18) + 1234
    words, _ = synth.many_criteria(13, 40, r)
    p = Pair(words, r)
    for T in (1, 2, 3, 7, 20, 39, 40, 41):
        p.check(list(range(40)), T, POS)
    rng = np.random.default_rng(14)
    ids = rng.integers(0, 40, size=300).tolist()
    for T in (1, 5, 60, 150, 299):
        p.check(ids, T, POS)


def test_position_many_criteria_full_size(many_criteria_full):
    words, r = many_criteria_full
    p = Pair(words, r)
    for T in (*synth.MANY_TS, 1, 64):
        p.check(list(range(synth.MANY_N)), T, POS)


# ---- the split-input kernel (the CTA's warps share a subtile's inputs)

SPLIT = thr.THR_VARIANT_SPLIT


def test_split_random_tiny_all_thresholds():
    rng = np.random.default_rng(404)
    for _ in range(20):
        n = int(rng.integers(1, 13))
        r = int(rng.choice([1, 63, 64, 65, 1000, 4096, 9000, 40000]))
        p = from_ints(oracle_pins.random_bitsets(rng, n, r), r)
        for T in range(0, n + 2):
            p.check(list(range(n)), T, SPLIT)


def test_split_many_inputs_and_chunks():
    """Fewer inputs than warps, and parts above one record chunk (n > 512)."""
    r = (1 << 17) + 999
    words, _ = synth.many_criteria(15, 40, r)
    p = Pair(words, r)
    for ids in ([3], [0, 7], [1, 2, 3], list(range(40))):
        for T in sorted({0, 1, 2, len(ids), len(ids) + 1}):
            p.check(ids, T, SPLIT)
    rng = np.random.default_rng(16)
    ids = rng.integers(0, 40, size=700).tolist()
    for T in (1, 3, 100, 350, 690, 700):
        p.check(ids, T, SPLIT)  # S > 8 for the middle thresholds: carry-save runs


def test_split_many_criteria_full_size(many_criteria_full):
    words, r = many_criteria_full
    p = Pair(words, r)
    for T in (*synth.MANY_TS, 1, 64):
        p.check(list(range(synth.MANY_N)), T, SPLIT)


# ---- the staged kernel's copies: stream segments that start at odd
#      and even stream words, sparse inputs packed several to a ring slot,
#      and the last words of the index

def test_staged_segments_alignment_and_index_end():
    r = (1 << 16) * 64 + 5  # W even + 1: the streams' parities alternate
    rng = np.random.default_rng(707)
    arrays = []
    for k in range(12):
        if k % 3 == 0:  # every word a literal: literal-run subtiles
            w = rng.integers(1, 1 << 62, size=synth.nwords(r), dtype=np.int64).astype(np.uint64)
            w[-1] &= np.uint64((1 << (r % 64)) - 1)
            w[-1] |= np.uint64(1)
            arrays.append(w)
        elif k % 3 == 1:
            arrays.append(synth.bernoulli(707, k, r, 3e-4))
        else:
            arrays.append(synth.clustered(707, k, r, 0.02))
    # the last bitmap: dense to its very last word (the end of the index)
    w = rng.integers(1, 1 << 62, size=synth.nwords(r), dtype=np.int64).astype(np.uint64)
    w[-1] = np.uint64((1 << (r % 64)) - 1) & np.uint64(0b10101)
    arrays.append(w)
    p = Pair(arrays, r)
    n = len(arrays)
    for T in (1, 2, 3, 4, 5, 7, n):
        for flags in (0, thr.THR_VARIANT_STAGED):
            p.check(list(range(n)), T, flags)
            p.check(list(range(n))[::-1] + [n - 1, 0], T, flags)


# ---- the staged carry-save kernel (inputs copied to shared memory first)

STAGED = thr.THR_VARIANT_STAGED


def test_staged_random_tiny_all_thresholds():
    rng = np.random.default_rng(505)
    for _ in range(20):
        n = int(rng.integers(1, 13))
        r = int(rng.choice([1, 63, 64, 65, 1000, 4096, 9000, 40000]))
        p = from_ints(oracle_pins.random_bitsets(rng, n, r), r)
        for T in range(0, n + 2):
            p.check(list(range(n)), T, STAGED)


def test_staged_many_criteria_full_size(many_criteria_full):
    words, r = many_criteria_full
    p = Pair(words, r)
    for T in (*synth.MANY_TS, 1, 64):
        p.check(list(range(synth.MANY_N)), T, STAGED)


# ---- the Looped levels (Algorithm 3, Sec. 6.2) for T <= 4

LOOPED = thr.THR_VARIANT_LOOPED


def test_looped_random_tiny_all_thresholds():
    rng = np.random.default_rng(606)
    for _ in range(20):
        n = int(rng.integers(1, 13))
        r = int(rng.choice([1, 63, 64, 65, 1000, 9000, 40000]))
        p = from_ints(oracle_pins.random_bitsets(rng, n, r), r)
        ids = rng.integers(0, n, int(rng.integers(1, 2 * n + 1))).tolist()
        for T in range(0, len(ids) + 2):  # T > 4 and T > n fall back to carry-save
            p.check(ids, T, LOOPED)


def test_looped_several_tiles_chunks_and_full_size(many_criteria_full):
    r = (1 << 18) + 3
    words, _ = synth.many_criteria(19, 30, r)
    p = Pair(words, r)
    rng = np.random.default_rng(20)
    for ids in (list(range(30)), rng.integers(0, 30, size=300).tolist()):
        for T in (1, 2, 3, 4, 5):
            p.check(ids, T, LOOPED)
    words, r = many_criteria_full
    p = Pair(words, r)
    for T in (1, 2, 3, 4):
        p.check(list(range(synth.MANY_N)), T, LOOPED)
    # in a batch, next to carry-save queries
    qs = [(list(range(synth.MANY_N)), T) for T in (2, 4, 16)]
    off, ln, pool = thr.thr_query_batch(p.g, qs, flags=LOOPED)
    for k, (ids, T) in enumerate(qs):
        assert np.array_equal(pool[int(off[k]): int(off[k] + ln[k])], p.o.threshold(ids, T))


# ---- symmetric functions of the counts: ranges and odd counts

def _check_sym(p, ids, lo, hi, odd=False):
    got = thr.thr_query_sym(p.g, ids, lo, hi, odd=odd)
    want = p.o.symmetric(ids, lo, hi, odd)
    assert np.array_equal(got, want), f"ids n={len(ids)} lo={lo} hi={hi} odd={odd}"


def test_symmetric_random_tiny_every_range():
    rng = np.random.default_rng(505)
    for _ in range(12):
        n = int(rng.integers(1, 9))
        r = int(rng.choice([1, 63, 64, 65, 1000, 9000, 40000]))
        p = from_ints(oracle_pins.random_bitsets(rng, n, r), r)
        ids = rng.integers(0, n, int(rng.integers(1, 2 * n + 1))).tolist()
        for lo in range(0, len(ids) + 2):
            for hi in range(lo, len(ids) + 2):
                _check_sym(p, ids, lo, hi)
        _check_sym(p, ids, 0, 0, odd=True)


def test_symmetric_several_tiles_and_chunks():
    r = (1 << 18) + 77
    words, _ = synth.many_criteria(17, 30, r)
    p = Pair(words, r)
    ids = list(range(30))
    for lo, hi in ((0, 0), (0, 2), (1, 1), (2, 5), (3, 30), (10, 12), (29, 29), (31, 40)):
        _check_sym(p, ids, lo, hi)
    _check_sym(p, ids, 0, 0, odd=True)
    rng = np.random.default_rng(18)
    ids = rng.integers(0, 30, size=300).tolist()  # n > 128: record chunks
    for lo, hi in ((0, 3), (5, 20), (40, 300)):
        _check_sym(p, ids, lo, hi)
    _check_sym(p, ids, 0, 0, odd=True)


def test_symmetric_many_criteria_full_size(many_criteria_full):
    words, r = many_criteria_full
    p = Pair(words, r)
    ids = list(range(synth.MANY_N))
    for lo, hi in ((0, 1), (1, 1), (2, 4), (5, 64)):
        _check_sym(p, ids, lo, hi)
    _check_sym(p, ids, 0, 0, odd=True)


# ---- a staged copy that never arrives: the bounded wait gives up

def test_lost_copy_returns_timeout_and_context_survives(monkeypatch):
    """Host-side fault injection: with THR_TEST_LOST_COPY=1 every ring slot
    waits for 16 bytes that are never sent.  The warp's wait gives up after
    about a second, the call returns THR_E_TIMEOUT, and the same query then
    runs exactly (the context is still usable)."""
    r = 640
    rng = np.random.default_rng(808)
    p = from_ints(oracle_pins.random_bitsets(rng, 3, r), r)
    monkeypatch.setenv("THR_TEST_LOST_COPY", "1")
    dense = [oracle_pins.mask(r) & int(x) for x in (0x5555 << 8, 0xF0F0F0F0F0F0F0F0F0F0)]
    q = from_ints(dense + [oracle_pins.mask(r) & 0x123456789ABCDEF], r)
    with pytest.raises(thr.ThrError) as e:
        thr.thr_query(q.g, [0, 1, 2], 2, flags=thr.THR_VARIANT_STAGED)
    assert e.value.status == thr.THR_E_TIMEOUT
    monkeypatch.delenv("THR_TEST_LOST_COPY")
    q.check([0, 1, 2], 2, thr.THR_VARIANT_STAGED)
    p.check([0, 1, 2], 2, thr.THR_VARIANT_STAGED)


def test_rows_past_two_to_the_26():
    """r past 2^26 rows (8288 subtiles, 33 pass-B scan blocks per query):
    single queries and a batch of several slots over clustered, i.i.d.,
    very sparse and tail-only bitmaps."""
    r = (1 << 26) + 777_777
    arrays = [synth.bernoulli(47, 0, r, 0.02), synth.clustered(47, 1, r, 0.3),
              synth.bernoulli(47, 2, r, 0.2), synth.clustered(47, 3, r, 0.05),
              synth.rows_to_words(np.arange(r - 5000, r), r), synth.bernoulli(47, 5, r, 1e-4)]
    p = Pair(arrays, r)
    assert (synth.nwords(r) + 127) // 128 > 8192
    for T in (1, 2, 3, 4):
        p.check(list(range(6)), T)
    qs = [(np.arange(6, dtype=np.uint32), T) for T in (1, 2, 3)]
    qs += [(np.array([1, 3, 4], np.uint32), 2), (np.array([0, 0, 2, 5], np.uint32), 2)]
    off, ln, pool = thr.thr_query_batch(p.g, qs, flags=thr.THR_NO_SHARE)
    for k, (ids, T) in enumerate(qs):
        assert np.array_equal(pool[int(off[k]): int(off[k] + ln[k])], p.o.threshold(ids, T)), k
