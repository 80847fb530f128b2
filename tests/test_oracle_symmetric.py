"""Pins of the oracle's symmetric-function queries (orc_symmetric): rows whose
count c over the ids satisfies lo <= c <= hi, or whose c is odd.  Checked
against brute force on tiny inputs (per-row counts from the uncompressed
bits), the XOR of the uncompressed words (odd counts), and set identities
with the threshold oracle: [T, n] is thr_T, [lo, hi] is thr_lo minus
thr_(hi+1), at most T is the complement of thr_(T+1), exactly k is
thr_k minus thr_(k+1)."""
import numpy as np
import pytest

import oracle
import oracle_pins
import synth


def _index(bitsets, r):
    """Bitmaps given as Python-integer bitsets (bit x = row x)."""
    words = [synth.rows_to_words(np.array([i for i in range(r) if (b >> i) & 1], dtype=np.int64),
                                 r) for b in bitsets]
    streams = [oracle.encode(w, r) for w in words]
    return oracle.Index(streams, r), words


def _rows(stream, r):
    return set(oracle.decode(stream, r).tolist())


def test_brute_force_tiny_every_range():
    rng = np.random.default_rng(77)
    for _ in range(25):
        n = int(rng.integers(1, 9))
        r = int(rng.choice([1, 63, 64, 65, 200, 1000]))
        bitsets = oracle_pins.random_bitsets(rng, n, r)
        o, words = _index(bitsets, r)
        ids = rng.integers(0, n, int(rng.integers(1, 2 * n + 1))).tolist()
        count = np.zeros(r, dtype=np.int64)
        for i in ids:
            count += synth.words_to_bits(words[i], r)
        for lo in range(0, len(ids) + 2):
            for hi in range(lo, len(ids) + 2):
                want = set(np.nonzero((count >= lo) & (count <= hi))[0].tolist())
                assert _rows(o.symmetric(ids, lo, hi), r) == want, (ids, lo, hi)
        want_odd = set(np.nonzero(count % 2 == 1)[0].tolist())
        assert _rows(o.symmetric(ids, 0, 0, odd=True), r) == want_odd


def test_odd_count_is_the_xor_of_the_inputs():
    r = 70_000
    words = [synth.bernoulli(3, k, r, p) for k, p in enumerate((0.01, 0.2, 0.5, 0.05, 0.3))]
    o = oracle.Index([oracle.encode(w, r) for w in words], r)
    x = np.bitwise_xor.reduce(np.stack(words), axis=0)
    assert np.array_equal(o.symmetric([0, 1, 2, 3, 4], 0, 0, odd=True), oracle.encode(x, r))
    # a repeated id cancels itself
    x2 = words[1] ^ words[2]
    assert np.array_equal(o.symmetric([0, 1, 2, 0], 0, 0, odd=True), oracle.encode(x2, r))


@pytest.mark.parametrize("seed", [1, 2])
def test_identities_with_thresholds(seed):
    r = 50_003
    words, _ = synth.many_criteria(seed, 10, r)
    o = oracle.Index([oracle.encode(w, r) for w in words], r)
    ids = list(range(10)) + [3, 3]
    n = len(ids)
    allrows = set(range(r))
    thr = {T: _rows(o.threshold(ids, T), r) for T in range(0, n + 2)}
    for T in range(0, n + 2):
        assert _rows(o.symmetric(ids, T, n), r) == thr[T]                     # [T, n]
        assert _rows(o.symmetric(ids, 0, T), r) == allrows - thr[T + 1] if T + 1 in thr \
            else _rows(o.symmetric(ids, 0, T), r) == allrows               # at most T
        if T + 1 in thr:
            assert _rows(o.symmetric(ids, T, T), r) == thr[T] - thr[T + 1]  # exactly T
    for lo, hi in ((1, 3), (2, 2), (4, 9), (0, 5), (6, 12)):
        assert _rows(o.symmetric(ids, lo, hi), r) == thr[lo] - thr.get(hi + 1, set())


SYM_MUTANTS = [
    ("upper bound exclusive", "count[x] >= lo && count[x] <= hi", "count[x] >= lo && count[x] < hi"),
    ("lower bound exclusive", "count[x] >= lo && count[x] <= hi", "count[x] > lo && count[x] <= hi"),
    ("parity inverted", "(int)(count[x] & 1u)", "(int)(~count[x] & 1u)"),
    ("bounds swapped", "count[x] >= lo && count[x] <= hi", "count[x] >= hi && count[x] <= lo"),
]


@pytest.mark.parametrize("name,old,new", SYM_MUTANTS, ids=[m[0] for m in SYM_MUTANTS])
def test_brute_force_kills_symmetric_mutants(tmp_path, name, old, new):
    src = open(oracle.SRC).read()
    assert old in src, f"mutation site for '{name}' no longer in oracle.c"
    c = tmp_path / "mutant.c"
    c.write_text(src.replace(old, new))
    lib = oracle.load(oracle.compile_c(str(c), str(tmp_path / "libmutant.so")))
    rng = np.random.default_rng(5)
    for _ in range(10):
        n, r = int(rng.integers(1, 6)), int(rng.choice([64, 130, 700]))
        bitsets = oracle_pins.random_bitsets(rng, n, r)
        words = [synth.rows_to_words(np.array([i for i in range(r) if (b >> i) & 1],
                                              dtype=np.int64), r) for b in bitsets]
        o = oracle.Index([oracle.encode(w, r) for w in words], r, lib=lib)
        ids = list(range(n)) * 2
        count = sum(synth.words_to_bits(w, r).astype(np.int64) for w in words) * 2
        for lo, hi, odd in ((1, 2, False), (0, 0, False), (2, 2 * n, False), (0, 0, True)):
            got = set(oracle.decode(o.symmetric(ids, lo, hi, odd), r).tolist())
            sel = (count % 2 == 1) if odd else (count >= lo) & (count <= hi)
            if got != set(np.nonzero(sel)[0].tolist()):
                return  # killed
    pytest.fail(f"mutant '{name}' survived")
