"""The opt-threshold profiling pass as an algorithm (no GPU): a plain
restatement of what each subtile does — skip when k + d cannot reach the
current lower bound, else walk the counts from its maximum down, add each
exact-count bin and raise the bound to a count the subtile alone shows on K
rows — run over the subtiles in many random orders, with and without a
seeding pass, must always give the oracle's answer.  This checks the claim the
kernel relies on: whatever order the warps take the subtiles in, the
histogram's suffix sums are exact down to the answer."""
import numpy as np
import pytest

import oracle
import synth

SUB = 8192  # rows per 128-word subtile


def _profile(counts, k_of, d_of, n, K, order, seed_stride=0):
    """Histogram and bound after one pass in `order` (and an optional
    seeding pass over every seed_stride-th subtile that only raises the
    bound); n inputs, so counts lie in 0..n."""
    hist = np.zeros(n + 1, np.int64)
    lb = 1

    def visit(g, record):
        nonlocal lb
        c = counts[g]
        k, d = k_of[g], d_of[g]
        L = lb
        if k + d < L:
            return
        if d == 0:
            if record:
                hist[k] += c.size
            if c.size >= K:
                lb = max(lb, k)
            return
        mx = int(c.max()) - k
        lo = max(L - k, 0)
        prev = 0
        for a in range(mx, lo - 1, -1):
            cnt = int((c >= k + a).sum())
            if record and cnt > prev:
                hist[k + a] += cnt - prev
            prev = cnt
            if cnt >= K:
                lb = max(lb, k + a)
                break

    if seed_stride:
        for g in range(0, len(counts), seed_stride):
            visit(g, False)
    for g in order:
        visit(g, True)
    return hist


def _answer(hist, n, K):
    atleast = 0
    for c in range(n, 0, -1):
        atleast += hist[c]
        if atleast >= K:
            return c
    return 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_any_subtile_order_gives_the_oracle_answer(seed):
    r = 24 * SUB + 100
    n_bm = 20
    words, _ = synth.many_criteria(seed, n_bm, r)
    bits = np.stack([synth.words_to_bits(w, r) for w in words]).astype(np.int64)
    rng = np.random.default_rng(seed)
    ids = rng.integers(0, n_bm, 30)
    rows = bits[ids].sum(axis=0)
    o = oracle.Index([oracle.encode(w, r) for w in words], r)
    ng = (r + SUB - 1) // SUB
    counts, k_of, d_of = [], [], []
    for g in range(ng):
        sl = slice(g * SUB, min((g + 1) * SUB, r))
        blk = bits[ids, sl]
        full = blk.all(axis=1)                 # ones fill over the subtile
        empty = ~blk.any(axis=1)               # zero fill
        counts.append(rows[sl])
        k_of.append(int(full.sum()))
        d_of.append(int((~full & ~empty).sum()))
    for K in (1, 2, 50, 3000, 10 ** 6):
        want, _ = o.opt_threshold(ids.tolist(), K)
        for trial in range(6):
            order = rng.permutation(ng)
            hist = _profile(counts, k_of, d_of, len(ids), K, order,
                            seed_stride=4 if trial % 2 else 0)
            assert _answer(hist, len(ids), K) == want, (K, trial)


def test_every_counted_row_matters_when_the_answer_is_one():
    """Sparse inputs where many subtiles hold a single active input: with K
    equal to the number of rows counted at least once the answer is 1, and
    with one more row it is 0 — a pass that skipped the subtiles whose counts
    can only equal the starting bound would answer 0 for the first."""
    r = 40 * SUB
    rng = np.random.default_rng(3)
    n_bm = 6
    bits = np.zeros((n_bm, r), np.int64)
    for g in range(40):  # one or two sparse inputs per subtile
        for b in rng.choice(n_bm, size=int(rng.integers(1, 3)), replace=False):
            rows = rng.choice(SUB, size=int(rng.integers(1, 40)), replace=False) + g * SUB
            bits[b, rows] = 1
    words = [synth.rows_to_words(np.nonzero(bits[b])[0], r) for b in range(n_bm)]
    o = oracle.Index([oracle.encode(w, r) for w in words], r)
    ids = np.arange(n_bm)
    rows = bits.sum(axis=0)
    counts, k_of, d_of = [], [], []
    for g in range(40):
        sl = slice(g * SUB, (g + 1) * SUB)
        blk = bits[:, sl]
        counts.append(rows[sl])
        k_of.append(0)
        d_of.append(int(blk.any(axis=1).sum()))
    ones = int((rows >= 1).sum())
    for K in (ones, ones + 1):
        want, _ = o.opt_threshold(ids.tolist(), K)
        assert want == (1 if K == ones else 0)
        for trial in range(4):
            hist = _profile(counts, k_of, d_of, n_bm, K, rng.permutation(40),
                            seed_stride=4 if trial % 2 else 0)
            assert _answer(hist, n_bm, K) == want, (K, trial)
