"""CPU model of the canonical re-encoding's aggregate monoid (the result words
of a query turned back into a marker/literal stream, Sec. 3.1 format).

Restated here from the library's definition: every result word has a class
(0 zero fill, 1 ones fill, 2 literal); a word starts a marker group when it is
a fill word following a literal or a fill of the other value, and word 0
always starts the first group.  A range of words is summarised by an
aggregate (heads after its first word, literals, the last head and the
literals before it, the first / last / last-head classes), and aggregates of
adjacent ranges combine associatively.  The GPU computes them per 128-word
subtile (pass A), scans them per block of 256 subtiles with 8 per lane and
the lanes' totals across the warp, then scans the block totals (pass B).

What is checked, against the oracle's own canonical encoder: the monoid is
associative; the blocked decomposition gives every subtile the same prefix as
a plain left-to-right scan; the whole result's heads + literals equal the
length of the oracle's encoding, and the last group's marker built from the
aggregate (pass B's final marker) equals the oracle's last marker.  Planted
mistakes in the model (the first word counted as a head, a fill after a
fill of the same value starting a group) are caught."""
import numpy as np
import pytest

import oracle
import synth

ALL = np.uint64(0xFFFFFFFFFFFFFFFF)


def classes(words):
    w = np.asarray(words, dtype=np.uint64)
    c = np.full(len(w), 2, dtype=np.int64)
    c[w == 0] = 0
    c[w == ALL] = 1
    return c.tolist()


def starts_group(prev, c, same_fill_starts=False):
    if c == 2:
        return False
    return prev == 2 or prev != c or same_fill_starts


# aggregate: (start, nh, nl, lh, lp, fc, lc, lhc, has)
def word_agg(x, c):
    return (x, 0, 1 if c == 2 else 0, 0, 0, c, c, 0, 0)


def combine(X, Y, same_fill_starts=False):
    xs, xnh, xnl, xlh, xlp, xfc, xlc, xlhc, xhas = X
    ys, ynh, ynl, ylh, ylp, yfc, ylc, ylhc, yhas = Y
    hf = starts_group(xlc, yfc, same_fill_starts)
    nh = xnh + (1 if hf else 0) + ynh
    nl = xnl + ynl
    if yhas:
        lh, lp, lhc, has = ylh, xnl + ylp, ylhc, 1
    elif hf:
        lh, lp, lhc, has = ys, xnl, yfc, 1
    else:
        lh, lp, lhc, has = xlh, xlp, xlhc, xhas
    return (xs, nh, nl, lh, lp, xfc, ylc, lhc, has)


def fix_first(a):
    s, nh, nl, lh, lp, fc, lc, lhc, has = a
    if not has:
        lh, lp, lhc, has = s, 0, fc, 1
    return (s, nh + 1, nl, lh, lp, fc, lc, lhc, has)


def fold(cls, x0, x1, **kw):
    a = word_agg(x0, cls[x0])
    for x in range(x0 + 1, x1):
        a = combine(a, word_agg(x, cls[x]), **kw)
    return a


def direct(cls, x0, x1, first_counts=False):
    """The aggregate of [x0, x1) computed from its definition, word by word."""
    heads = [x for x in range(x0 + 1, x1) if starts_group(cls[x - 1], cls[x])]
    if first_counts:
        heads = [x0] + heads
    nl = sum(1 for x in range(x0, x1) if cls[x] == 2)
    if heads:
        lh = heads[-1]
        lp = sum(1 for x in range(x0, lh) if cls[x] == 2)
        lhc, has = cls[lh], 1
    else:
        lh = lp = lhc = has = 0
    return (x0, len(heads), nl, lh, lp, cls[x0], cls[x1 - 1], lhc, has)


def random_words(rng, W, r):
    """Words with long fills of both values, literals, and runs of each."""
    out = np.zeros(W, dtype=np.uint64)
    x = 0
    while x < W:
        kind = rng.integers(0, 4)
        n = int(rng.integers(1, 40))
        if kind == 0:
            out[x:x + n] = 0
        elif kind == 1:
            out[x:x + n] = ALL
        else:
            out[x:x + n] = rng.integers(1, 1 << 62, size=len(out[x:x + n]),
                                        dtype=np.int64).astype(np.uint64)
        x += n
    if r % 64:
        out[-1] &= np.uint64((1 << (r % 64)) - 1)
    return out


def test_word_fold_equals_definition_and_is_associative():
    rng = np.random.default_rng(11)
    for _ in range(60):
        W = int(rng.integers(2, 300))
        cls = classes(random_words(rng, W, 64 * W))
        assert fold(cls, 0, W) == direct(cls, 0, W)
        a, b, c = sorted(rng.choice(np.arange(1, W), size=3, replace=True).tolist()) if W > 3 else (1, 1, 1)
        if not (0 < a < b < c < W):
            continue
        A, B, C, D = fold(cls, 0, a), fold(cls, a, b), fold(cls, b, c), fold(cls, c, W)
        left = combine(combine(combine(A, B), C), D)
        right = combine(A, combine(B, combine(C, D)))
        assert left == right == direct(cls, 0, W)


@pytest.mark.parametrize("sub,per_lane,lanes", [(128, 8, 32), (4, 2, 4), (3, 3, 2)])
def test_blocked_scan_gives_every_subtile_its_prefix(sub, per_lane, lanes):
    """Subtile aggregates (sub words), blocks of per_lane * lanes subtiles
    scanned lane-locally then across the lanes, then the block totals scanned
    in order: every subtile's prefix equals the plain scan of the words
    before it (word 0's group counted)."""
    rng = np.random.default_rng(12 + sub)
    for _ in range(8):
        W = int(rng.integers(1, 40 * sub))
        cls = classes(random_words(rng, W, 64 * W))
        NG = -(-W // sub)
        aggs = [fold(cls, g * sub, min(W, (g + 1) * sub)) for g in range(NG)]
        aggs[0] = fix_first(aggs[0])
        blk = per_lane * lanes
        NB = -(-NG // blk)
        pref = [None] * NG
        totals = []
        for b in range(NB):
            lane_tot = []
            for ln in range(lanes):
                run = None
                for i in range(per_lane):
                    g = b * blk + ln * per_lane + i
                    if g < NG:
                        run = aggs[g] if run is None else combine(run, aggs[g])
                lane_tot.append(run)
            # exclusive prefix of each lane, then of each subtile in the lane
            E = None
            for ln in range(lanes):
                e = E
                for i in range(per_lane):
                    g = b * blk + ln * per_lane + i
                    if g < NG:
                        pref[g] = e
                        e = aggs[g] if e is None else combine(e, aggs[g])
                if lane_tot[ln] is not None:
                    E = lane_tot[ln] if E is None else combine(E, lane_tot[ln])
            totals.append(E)
        carry = None
        bpref = []
        for t in totals:
            bpref.append(carry)
            carry = t if carry is None else combine(carry, t)
        for g in range(1, NG):
            b = g // blk
            inb, bp = pref[g], bpref[b]
            P = bp if inb is None else (inb if bp is None else combine(bp, inb))
            assert P == direct(cls, 0, g * sub, first_counts=True), (g, b)
        assert carry == direct(cls, 0, W, first_counts=True)


def final_marker(a, W):
    """Pass B's marker of the result's last group, from the whole aggregate."""
    _, nh, nl, lh, lp, _, _, lhc, _ = a
    L = nl - lp
    F = W - lh - L
    bit = 1 if (F and lhc == 1) else 0
    return nh - 1 + lp, bit | (F << 1) | (L << 33)


@pytest.mark.parametrize("kind", ["random", "bernoulli", "clustered", "empty", "full"])
def test_whole_aggregate_matches_the_oracle_encoding(kind):
    rng = np.random.default_rng({"random": 1, "bernoulli": 2, "clustered": 3,
                                 "empty": 4, "full": 5}[kind])
    for _ in range(12):
        r = int(rng.integers(1, 64 * 400))
        W = synth.nwords(r)
        if kind == "random":
            words = random_words(rng, W, r)
        elif kind == "bernoulli":
            words = synth.bernoulli(int(rng.integers(1 << 30)), 0, r, float(rng.uniform(1e-3, 0.2)))
        elif kind == "clustered":
            words = synth.clustered(int(rng.integers(1 << 30)), 0, r, float(rng.uniform(0.01, 0.5)))
        elif kind == "empty":
            words = np.zeros(W, dtype=np.uint64)
        else:
            words = synth.rows_to_words(np.arange(r), r)
        stream = oracle.encode(words, r)
        a = fix_first(fold(classes(words), 0, W))
        assert a[1] + a[2] == len(stream)
        pos, marker = final_marker(a, W)
        assert int(stream[pos]) == marker


def test_planted_mistakes_are_caught():
    rng = np.random.default_rng(99)
    words = random_words(rng, 300, 64 * 300)
    cls = classes(words)
    stream = oracle.encode(words, 64 * 300)
    # counting word 0 without fix_first, or as a head inside its range
    plain = fold(cls, 0, 300)
    assert plain[1] + plain[2] != len(stream)
    # a fill after a fill of the same value starting a new group
    wrong = fix_first(fold(cls, 0, 300, same_fill_starts=True))
    assert wrong[1] + wrong[2] != len(stream)
