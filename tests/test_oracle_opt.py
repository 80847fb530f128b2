"""Pins of the oracle's opt-threshold query (orc_opt_threshold): the largest T
whose T-overlap result holds at least K rows, and that result.  Checked
against brute force over per-row counts from the uncompressed bits, the
descending search of Barbay and Kenyon (Sec. 5.2: try T = n, n - 1, ...
with the threshold oracle until K rows come back), the Looped route of
Sec. 6.2 (run Algorithm 3 with T = n and take the largest i whose C_i holds
K rows), invariants in K, and planted mistakes that these checks catch."""
import numpy as np
import pytest

import oracle
import oracle_pins
import synth


def _index(bitsets, r, lib=None):
    words = [oracle_pins.int_to_words(b, r) for b in bitsets]
    return oracle.Index([oracle.encode(w, r) for w in words], r, lib=lib), words


def _rows(stream, r):
    return set(oracle.decode(stream, r).tolist())


def _counts(bitsets, ids, r):
    return np.array([sum((bitsets[i] >> x) & 1 for i in ids) for x in range(r)], dtype=np.int64)


def test_brute_force_tiny_every_k():
    rng = np.random.default_rng(91)
    for _ in range(30):
        n = int(rng.integers(1, 8))
        r = int(rng.choice([1, 5, 63, 64, 65, 130, 400]))
        bitsets = oracle_pins.random_bitsets(rng, n, r)
        o, _ = _index(bitsets, r)
        ids = rng.integers(0, n, int(rng.integers(1, 2 * n + 1))).tolist()
        count = _counts(bitsets, ids, r)
        for K in list(range(1, min(r, 12) + 1)) + [r, r + 1, r + 7]:
            T_bf = 0
            for T in range(0, len(ids) + 1):
                if int((count >= T).sum()) >= K:
                    T_bf = T
            T, s = o.opt_threshold(ids, K)
            assert T == T_bf, (ids, K)
            assert _rows(s, r) == set(np.nonzero(count >= T_bf)[0].tolist())
        # K = 1: the largest count, and exactly the rows that reach it
        T, s = o.opt_threshold(ids, 1)
        assert T == int(count.max())
        assert _rows(s, r) == set(np.nonzero(count == count.max())[0].tolist())


def test_descending_search_and_looped_agree():
    rng = np.random.default_rng(5)
    for _ in range(12):
        n = int(rng.integers(2, 10))
        r = int(rng.choice([64, 200, 1000, 3000]))
        bitsets = oracle_pins.random_bitsets(rng, n, r)
        o, _ = _index(bitsets, r)
        ids = list(range(n))
        _, C = oracle_pins.looped(bitsets, n)
        for K in (1, 2, 5, 17, r // 3, r):
            # Sec. 5.2: T = n, n - 1, ... until the result holds K rows
            T_desc = 0
            for T in range(n, 0, -1):
                if len(oracle.decode(o.threshold(ids, T), r)) >= K:
                    T_desc = T
                    break
            # Sec. 6.2: Looped's C_i holds the rows counted at least i times
            T_loop = max([i for i in range(1, n + 1) if bin(C[i]).count("1") >= K], default=0)
            T, s = o.opt_threshold(ids, K)
            assert T == T_desc == T_loop, (n, r, K)
            assert np.array_equal(s, o.threshold(ids, T))


def test_monotone_in_k_and_tight():
    r = 40_000
    words, _ = synth.many_criteria(4, 12, r)
    o = oracle.Index([oracle.encode(w, r) for w in words], r)
    ids = list(range(12)) + [2, 7]
    prev = None
    for K in (1, 2, 3, 10, 100, 1000, 10_000, r, r + 1):
        T, s = o.opt_threshold(ids, K)
        size = len(oracle.decode(s, r))
        assert size >= K or (K > r and T == 0 and size == r)
        if T < len(ids):
            assert len(oracle.decode(o.threshold(ids, T + 1), r)) < K  # T + 1 is too high
        if prev is not None:
            assert T <= prev  # a larger K never raises T
        prev = T


def test_no_qualifying_threshold_gives_every_row():
    r = 100
    o, _ = _index([0, 0], r)  # two empty bitmaps: every row counts 0
    T, s = o.opt_threshold([0, 1], 1)
    assert T == 0 and _rows(s, r) == set(range(r))
    o, _ = _index([(1 << r) - 1], r)  # one full bitmap
    assert o.opt_threshold([0, 0, 0], 1)[0] == 3
    assert o.opt_threshold([0, 0, 0], r)[0] == 3
    T, s = o.opt_threshold([0, 0, 0], r + 1)
    assert T == 0 and _rows(s, r) == set(range(r))


def test_k_zero_is_rejected():
    o, _ = _index([1], 10)
    with pytest.raises(oracle.OracleError):
        o.opt_threshold([0], 0)


OPT_MUTANTS = [
    ("strict at-least test", "if (atleast >= K)", "if (atleast > K)"),
    ("search starts one below n", "for (uint32_t c = n; c >= 1; c--)",
     "for (uint32_t c = n - 1; c >= 1; c--)"),
    ("result keeps counts above T only", "            if (count[x] >= T) words",
     "            if (count[x] > T) words"),
    ("suffix sum skips the top bin", "            atleast += hist[c];\n            if",
     "            if (c < n) atleast += hist[c];\n            if"),
]


@pytest.mark.parametrize("name,old,new", OPT_MUTANTS, ids=[m[0] for m in OPT_MUTANTS])
def test_checks_kill_opt_mutants(tmp_path, name, old, new):
    src = open(oracle.SRC).read()
    assert src.count(old) == 1, f"mutation site for '{name}' not unique in oracle.c"
    c = tmp_path / "mutant.c"
    c.write_text(src.replace(old, new))
    lib = oracle.load(oracle.compile_c(str(c), str(tmp_path / "libmutant.so")))
    rng = np.random.default_rng(8)
    for _ in range(10):
        n, r = int(rng.integers(1, 6)), int(rng.choice([64, 130, 700]))
        bitsets = oracle_pins.random_bitsets(rng, n, r)
        o, _ = _index(bitsets, r, lib=lib)
        ids = list(range(n))
        count = _counts(bitsets, ids, r)
        for K in (1, 2, 3, r // 2):
            T_bf = max(T for T in range(0, n + 1) if int((count >= T).sum()) >= K)
            T, s = o.opt_threshold(ids, K)
            if T != T_bf or _rows(s, r) != set(np.nonzero(count >= T_bf)[0].tolist()):
                return  # killed
    pytest.fail(f"mutant '{name}' survived")


def test_count_histogram_brute_force_and_threshold_sizes():
    """The count histogram against per-row counts from the uncompressed bits
    (brute force) and, by suffix sums, against the sizes of the threshold
    oracle's results; bins add up over row shards cut at any word boundary."""
    rng = np.random.default_rng(93)
    for _ in range(25):
        n = int(rng.integers(1, 8))
        r = int(rng.choice([1, 5, 63, 64, 65, 130, 400, 1000]))
        bitsets = oracle_pins.random_bitsets(rng, n, r)
        o, words = _index(bitsets, r)
        ids = rng.integers(0, n, int(rng.integers(1, 2 * n + 1))).tolist()
        hist = o.count_histogram(ids)
        want = np.bincount(_counts(bitsets, ids, r), minlength=len(ids) + 1)
        assert hist.tolist() == want.tolist()
        for T in range(0, len(ids) + 2):
            size = len(_rows(o.threshold(ids, T), r))
            assert size == int(hist[T:].sum())
        W = (r + 63) // 64
        if W >= 2:
            cut = int(rng.integers(1, W))
            lo = [oracle.encode(w[:cut], 64 * cut) for w in words]
            hi = [oracle.encode(w[cut:], r - 64 * cut) for w in words]
            h = (oracle.Index(lo, 64 * cut).count_histogram(ids) +
                 oracle.Index(hi, r - 64 * cut).count_histogram(ids))
            assert h.tolist() == hist.tolist()
