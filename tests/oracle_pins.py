"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, never against the oracle itself.

Every ``pin_*`` function takes an ``oracle.Oracle`` (the real one, or a
deliberately mutated copy in ``test_oracle_mutants.py``) and raises
AssertionError when the oracle disagrees with

* the worked examples printed in Kaser & Lemire, arXiv 1402.4466 (fixtures
  under ``tests/golden/``, each citing its section);
* brute force (per-row counting over uncompressed bits) on tiny inputs;
* two independent algorithms written here from the paper over Python-integer
  bitsets: Looped (Algorithm 3, Sec. 6.2) and BSTM (Algorithm 2, Sec. 5.3.1);
* closed-form invariants: T = 1 is OR and T = N is AND (Sec. 2), results
  shrink as T grows, NOT(thr_T(B)) = thr_{N-T+1}(NOT B) (the at-most rewrite
  of Sec. 2), sum |B_i| >= T |result| (Sec. 2.1 lower bound), a duplicated id
  counts twice;
* hand-written canonical streams of the project's stream format and a list of
  malformed streams that must be rejected.
"""
from __future__ import annotations

import numpy as np

import oracle
from golden import (ALL_ONES, bits_row0_first, format_cases, hex_words,
                    marker, read_kv)

# ---------------------------------------------------------------- helpers


def nwords(r: int) -> int:
    return (r + 63) // 64


def int_to_words(x: int, r: int) -> np.ndarray:
    W = nwords(r)
    return np.array([(x >> (64 * i)) & ALL_ONES for i in range(W)],
                    dtype=np.uint64)


def words_to_int(words) -> int:
    return sum(int(w) << (64 * i) for i, w in enumerate(words))


def rows_of(x: int) -> list[int]:
    out, i = [], 0
    while x:
        if x & 1:
            out.append(i)
        x >>= 1
        i += 1
    return out


def mask(r: int) -> int:
    return (1 << r) - 1


def streams_for(o, bitsets, r):
    return [o.encode(int_to_words(b, r), r) for b in bitsets]


def query(o, bitsets, r, T, ids=None):
    """Oracle result of thr_T over the given bitsets, as a Python int, plus
    its encoded stream."""
    streams = streams_for(o, bitsets, r)
    words, offs = oracle.concat(streams)
    if ids is None:
        ids = list(range(len(bitsets)))
    enc = o.threshold(words, offs, r, ids, T)
    dec = o.decode(enc, r)
    as_int = sum(1 << int(x) for x in dec)
    w = o.threshold_words(words, offs, r, ids, T)
    assert words_to_int(w) == as_int, "encoded and word results differ"
    return as_int, enc


def brute(bitsets, r, T, ids=None):
    """Per-row count over uncompressed bits (the definition of Sec. 2)."""
    if ids is None:
        ids = list(range(len(bitsets)))
    count = np.zeros(r, dtype=np.int64)
    for i in ids:
        count += np.array([(bitsets[i] >> x) & 1 for x in range(r)],
                          dtype=np.int64)
    return sum(1 << int(x) for x in np.nonzero(count >= T)[0])


def looped(bitsets, T):
    """Algorithm 3 (Sec. 6.2): C_j <- C_j OR (C_{j-1} AND B_i), j = min(T,i)..2,
    then C_1 <- C_1 OR B_i; the answer is C_T.  Defined for 1 <= T <= N."""
    C = [0] * (T + 1)
    C[1] = bitsets[0]
    for i in range(2, len(bitsets) + 1):
        Bi = bitsets[i - 1]
        for j in range(min(T, i), 1, -1):
            C[j] = C[j] | (C[j - 1] & Bi)
        C[1] = C[1] | Bi
    return C[T], C


def bstm(bitsets, T, r):
    """Algorithm 2 (Sec. 5.3.1): ripple-add the inputs into bit slices A_1..,
    then compare the Hamming weights against T - 1 (greater than), slices
    from the most significant down.  Returns (answer, slices)."""
    N = len(bitsets)
    nsl = max(1, (2 * N).bit_length() - 1)  # floor(log2(2N))
    A = [0] * (nsl + 2)
    A[1] = bitsets[0]
    for i in range(2, N + 1):
        Bi = bitsets[i - 1]
        C = Bi & A[1]
        A[1] = Bi ^ A[1]
        j = 2
        while C:
            C, A[j] = C & A[j], C ^ A[j]
            j += 1
    full = mask(r)
    beq, bgt = full, 0
    t1 = T - 1
    for j in range(nsl, 0, -1):
        if (t1 >> (j - 1)) & 1:
            beq = beq & A[j]
        else:
            bgt = bgt | (beq & A[j])
            beq = beq & (~A[j] & full)
    return bgt, A


def random_bitsets(rng, n, r):
    """Tiny structured bitmaps: random bits, runs, all zeros, all ones and
    blocks of whole words (so that fills, literals and ragged tails occur)."""
    out = []
    W = nwords(r)
    for _ in range(n):
        kind = rng.integers(0, 6)
        if kind == 0:
            p = rng.choice([0.01, 0.1, 0.5, 0.9])
            x = sum(1 << i for i in np.nonzero(rng.random(r) < p)[0].tolist())
        elif kind == 1:
            x = 0
            pos = 0
            while pos < r:
                pos += int(rng.geometric(1 / 40))
                ln = int(rng.geometric(1 / 90))
                x |= mask(min(ln, max(r - pos, 0))) << pos if pos < r else 0
                pos += ln
        elif kind == 2:
            x = 0
        elif kind == 3:
            x = mask(r)
        else:
            x = 0
            for w in range(W):
                c = rng.integers(0, 4)
                if c == 1:
                    x |= ALL_ONES << (64 * w)
                elif c == 2:
                    x |= int(rng.integers(1, 1 << 62)) << (64 * w)
            x &= mask(r)
        out.append(x & mask(r))
    return out


# ------------------------------------------------------- worked examples


def pin_fig1(o):
    g = read_kv("fig1_threshold.txt")
    r, T = int(g["r"]), int(g["T"])
    B = [bits_row0_first(g[k]) for k in ("B1", "B2", "B3")]
    got, _ = query(o, B, r, T)
    assert got == bits_row0_first(g["result"]), "Fig. 1"


def pin_sets_example(o):
    g = read_kv("sets_example.txt")
    r = int(g["r"])
    S = [[int(v) for v in g[k].split()] for k in ("S1", "S2")]
    B = [sum(1 << v for v in s) for s in S]
    for b, k in zip(B, ("msb_first_1", "msb_first_2")):
        assert format(b, "08b") == g[k], "bit order (Sec. 2)"
    streams = streams_for(o, B, r)
    rows = [o.decode(s, r).tolist() for s in streams]
    assert rows == S, "decoded rows"
    assert sum(len(x) for x in rows) == int(g["B"]), "B = sum of cardinalities"
    assert query(o, B, r, 2)[0] == (B[0] & B[1])
    assert query(o, B, r, 1)[0] == (B[0] | B[1])


def pin_word_layout(o):
    g = read_kv("word_layout.txt")
    rows = [int(v) for v in g["rows"].split()]
    r = int(g["r"])
    w8 = [int(t, 2) for t in g["words_msb_first"].split()]
    # the 64-bit word holds the 8-bit words in order, lowest first
    w64 = sum(w << (8 * i) for i, w in enumerate(w8))
    assert w64 == sum(1 << v for v in rows)
    s = o.encode(np.array([w64], dtype=np.uint64), r)
    assert s.tolist() == [marker(0, 0, 1), w64], "one literal after a marker"
    assert o.decode(s, r).tolist() == rows


def pin_bstm_trace(o):
    g = read_kv("bstm_trace.txt")
    r, T = int(g["r"]), int(g["T"])
    B = [bits_row0_first(g[k]) for k in ("B1", "B2", "B3")]
    want = bits_row0_first(g["result"])
    ans, A = bstm(B, T, r)
    assert A[1] == bits_row0_first(g["A1"]) and A[2] == bits_row0_first(g["A2"])
    assert ans == want
    assert query(o, B, r, T)[0] == want, "BSTM illustration (Sec. 5.3.1)"


def pin_looped_trace(o):
    g = read_kv("looped_trace.txt")
    r, T = int(g["r"]), int(g["T"])
    B = [bits_row0_first(g[k]) for k in ("B1", "B2", "B3")]
    _, C2 = looped(B[:2], T)
    assert C2[1] == bits_row0_first(g["C1_after_B2"])
    assert C2[2] == bits_row0_first(g["C2_after_B2"])
    ans, C = looped(B, T)
    assert C[1] == bits_row0_first(g["C1"]) and C[2] == bits_row0_first(g["C2"])
    assert ans == bits_row0_first(g["result"])
    assert query(o, B, r, T)[0] == ans, "Looped illustration (Sec. 6.2)"


def pin_rbmrg_ewah(o):
    g = read_kv("rbmrg_ewah.txt")
    r, T = int(g["r"]), int(g["T"])
    B = [words_to_int(hex_words(g[k])) for k in ("B1", "B2", "B3", "B4")]
    want = words_to_int(hex_words(g["result"]))
    got, enc = query(o, B, r, T)
    assert got == want, "EWAH example (Sec. 6.4)"
    assert query(o, B, r, 1)[0] == (B[0] | B[1] | B[2] | B[3])
    assert query(o, B, r, 4)[0] == (B[0] & B[1] & B[2] & B[3])


# ------------------------------------------------------------ stream format


def pin_format_cases(o):
    for r, w, s in format_cases():
        words = np.array(w, dtype=np.uint64)
        got = o.encode(words, r).tolist()
        assert got == s, f"encode r={r} {w}: {got} != {s}"
        assert o.validate(np.array(s, dtype=np.uint64), r) == 0
        assert o.decode(np.array(s, dtype=np.uint64), r).tolist() == \
            rows_of(words_to_int(w))


def bad_streams():
    """(r, stream) pairs that break one canonical rule or the coverage."""
    m = marker
    O = ALL_ONES
    return [
        (128, [m(0, 1, 0), m(0, 1, 0)]),          # (ii) fill run split
        (128, [m(1, 1, 0), m(1, 1, 0)]),          # (ii) ones fill split
        (128, [m(0, 0, 2), 5, 0]),                # (i) literal 0
        (128, [m(0, 0, 2), 5, O]),                # (i) literal ~0
        (128, [m(1, 0, 2), 5, 6]),                # (iv) b = 1 with F = 0
        (128, [m(0, 0, 1), 5, m(0, 0, 1), 6]),    # (vi) F = 0 mid-stream
        (128, [m(0, 3, 0)]),                      # covers too much
        (192, [m(0, 2, 0)]),                      # covers too little
        (128, [m(0, 2, 0), 7]),                   # word after the end
        (128, [m(0, 0, 2), 5]),                   # truncated literals
        (100, [m(1, 2, 0)]),                      # (v) ones over ragged word
        (100, [m(0, 1, 1), 1 << 40]),             # (v) bit past r
        (64, [m(0, 0, 0), m(0, 1, 0)]),           # empty marker
        (0, [m(0, 1, 0)]),                        # r = 0 must be [0]
        (0, []),
    ]


def pin_rejects_malformed(o):
    for r, s in bad_streams():
        rc = o.validate(np.array(s, dtype=np.uint64), r)
        assert rc == oracle.E_FORMAT, f"accepted malformed r={r} {s}"


def pin_roundtrip(o, seed=7, trials=60):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        r = int(rng.choice([1, 63, 64, 65, 127, 128, 129, 640, 1000, 4096,
                            4097]))
        x = random_bitsets(rng, 1, r)[0]
        w = int_to_words(x, r)
        s = o.encode(w, r)
        assert o.validate(s, r) == 0
        assert len(s) <= nwords(r) + 1
        assert o.decode(s, r).tolist() == rows_of(x)


# ------------------------------------------------------ brute force & co


def pin_brute_force(o, seed=11, trials=25):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        n = int(rng.integers(1, 13))
        r = int(rng.choice([1, 5, 64, 65, 200, 511, 1024, 3001, 4096]))
        B = random_bitsets(rng, n, r)
        for T in range(0, n + 2):
            got, enc = query(o, B, r, T)
            want = brute(B, r, T)
            assert got == want, f"n={n} r={r} T={T}"
            assert enc.tolist() == o.encode(int_to_words(want, r), r).tolist()


def pin_independent_algorithms(o, seed=13, trials=20):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        n = int(rng.integers(1, 10))
        r = int(rng.choice([8, 64, 100, 130, 777, 2048]))
        B = random_bitsets(rng, n, r)
        for T in range(1, n + 1):
            got = query(o, B, r, T)[0]
            assert got == looped(B, T)[0], f"Looped n={n} T={T}"
            assert got == bstm(B, T, r)[0], f"BSTM n={n} T={T}"


def pin_invariants(o, seed=17, trials=15):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        n = int(rng.integers(2, 9))
        r = int(rng.choice([64, 65, 300, 1000, 1536]))
        B = random_bitsets(rng, n, r)
        full = mask(r)
        res = [query(o, B, r, T)[0] for T in range(0, n + 2)]
        orr, andd = 0, full
        for b in B:
            orr |= b
            andd &= b
        assert res[0] == full, "T = 0 selects every row"
        assert res[1] == orr, "T = 1 is OR"
        assert res[n] == andd, "T = N is AND"
        assert res[n + 1] == 0, "T > N selects nothing"
        for T in range(0, n + 1):
            assert res[T + 1] & ~res[T] == 0, "monotone in T"
        notB = [full & ~b for b in B]
        for T in range(1, n + 1):
            comp = query(o, notB, r, n - T + 1)[0]
            assert (full & ~res[T]) == comp, "NOT thr_T(B) = thr_{N-T+1}(NOT B)"
            assert sum(bin(b).count("1") for b in B) >= T * bin(res[T]).count("1")
        # a duplicated id counts twice
        dup = query(o, B, r, 2, ids=[0, 0])[0]
        assert dup == B[0], "duplicate ids count with multiplicity"
        dup3 = query(o, B, r, 3, ids=[0, 0, 1])[0]
        assert dup3 == (B[0] & B[1])


def pin_row_partitions(o, seed=19, trials=25):
    """The row-partitioned ScanCount (the multi-core CPU baseline) against
    brute force: every split of the rows into word ranges, including more
    ranges than words, fills of ones that cross range borders, ragged tails
    and repeated ids."""
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        n = int(rng.integers(1, 9))
        r = int(rng.choice([1, 64, 65, 300, 1000, 1536, 4097]))
        B = random_bitsets(rng, n, r)
        words, offs = oracle.concat(streams_for(o, B, r))
        ids = list(range(n)) + [int(rng.integers(0, n))]
        for parts in (1, 2, 3, 7, nwords(r) + 2):
            for T in range(0, n + 3):
                enc = o.threshold_parts(words, offs, r, ids, T, parts)
                want = brute(B, r, T, ids)
                got = sum(1 << int(x) for x in o.decode(enc, r))
                assert got == want, f"parts={parts} n={n} r={r} T={T}"
                assert enc.tolist() == o.encode(int_to_words(want, r), r).tolist()


ALL_PINS = [pin_fig1, pin_sets_example, pin_word_layout, pin_bstm_trace,
            pin_looped_trace, pin_rbmrg_ewah, pin_format_cases,
            pin_rejects_malformed, pin_roundtrip, pin_brute_force,
            pin_independent_algorithms, pin_invariants, pin_row_partitions]
