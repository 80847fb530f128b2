"""GPU parity of batched queries (thr_query_batch): every result of a batch
equals the CPU oracle's word for word and equals the same query run alone
through thr_query, whatever the batch around it: chunked batches, CUDA-graph
replay (a cached graph updated with new parameters), device and host pools,
an undersized pool, and every selection policy."""

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


def _index(word_arrays, r):
    gw, goff = thr.encode_many(word_arrays, r)
    ostreams = [oracle.encode(w, r) for w in word_arrays]
    ow, ooff = oracle.concat(ostreams)
    assert np.array_equal(gw, ow) and np.array_equal(goff, ooff)
    return thr.idx_build_rle(gw, goff, r), oracle.Index(ostreams, r)


@pytest.fixture(scope="module")
def mixed():
    """48 bitmaps over 3 tiles + a ragged tail: i.i.d. densities from 1e-4
    to 0.6, clustered runs, an empty and a full bitmap."""
    r = 3 * 8192 * 4 + 4100
    rng = np.random.default_rng(11)
    arrays = []
    for i in range(48):
        if i == 0:
            arrays.append(np.zeros(synth.nwords(r), np.uint64))
        elif i == 1:
            arrays.append(synth.rows_to_words(np.arange(r), r))
        elif i % 3 == 0:
            arrays.append(synth.clustered(11, i, r, float(10 ** rng.uniform(-3, -0.3))))
        else:
            arrays.append(synth.bernoulli(11, i, r, float(10 ** rng.uniform(-4, -0.2))))
    g, o = _index(arrays, r)
    return g, o, r


def _queries(seed, nb, nq, nmax=40):
    rng = np.random.default_rng(seed)
    qs = []
    for k in range(nq):
        n = int(rng.integers(1, nmax + 1))
        ids = rng.integers(0, nb, n).astype(np.uint32)  # with replacement
        T = int(rng.integers(0, n + 2))                  # 0 .. n + 1
        qs.append((ids, T))
    return qs


def _check(g, o, qs, off, ln, pool):
    for k, (ids, T) in enumerate(qs):
        got = np.asarray(pool[int(off[k]): int(off[k]) + int(ln[k])], dtype=np.uint64)
        want = o.threshold(ids, T)
        assert np.array_equal(got, want), f"query {k}: n={len(ids)} T={T}"
    # results lie back to back in query order
    assert off[0] == 0 and np.array_equal(off[1:], np.cumsum(ln)[:-1])


def test_batch_matches_oracle_host_pool(mixed):
    g, o, r = mixed
    qs = _queries(1, 48, 60)
    off, ln, pool = thr.thr_query_batch(g, qs)
    _check(g, o, qs, off, ln, pool)
    assert thr.thr_last_batch_info()["graph"] in (0, 1)


def test_batch_device_pool_and_no_graph_agree(mixed, cuda):
    g, o, r = mixed
    qs = _queries(2, 48, 40)
    pool = cuda.zeros(40 * (synth.nwords(r) + 1), dtype=cuda.int64, device="cuda")
    off, ln, _ = thr.thr_query_batch(g, qs, pool=pool)
    host = pool.cpu().numpy().view(np.uint64)
    _check(g, o, qs, off, ln, host)
    off2, ln2, pool2 = thr.thr_query_batch(g, qs, flags=thr.THR_NO_GRAPH)
    assert thr.thr_last_batch_info()["graph"] == -1
    assert np.array_equal(ln, ln2) and np.array_equal(off, off2)
    assert np.array_equal(host[: int(ln.sum())], pool2[: int(ln2.sum())])


def test_batch_equals_single_queries(mixed):
    g, o, r = mixed
    qs = _queries(3, 48, 25)
    off, ln, pool = thr.thr_query_batch(g, qs)
    for k, (ids, T) in enumerate(qs):
        alone = thr.thr_query(g, ids, T)
        assert np.array_equal(pool[int(off[k]): int(off[k]) + int(ln[k])], alone)


def test_batch_chunked(mixed, monkeypatch):
    """Scratch for 3 queries at a time: the chunks run one after another and
    place their results after the earlier chunks'."""
    g, o, r = mixed
    monkeypatch.setenv("THR_MAX_SLOTS", "3")
    qs = _queries(4, 48, 17)
    off, ln, pool = thr.thr_query_batch(g, qs)
    info = thr.thr_last_batch_info()
    assert info["chunks"] == 6
    _check(g, o, qs, off, ln, pool)
    off2, ln2, pool2 = thr.thr_query_batch(g, qs, flags=thr.THR_NO_GRAPH)
    assert np.array_equal(ln, ln2)


def test_graph_replayed_with_new_inputs(mixed):
    """Two batches of the same shape (same kernel classes per chunk) but other
    ids and thresholds: the second call updates and replays the cached graph,
    and its results are those of the new queries."""
    g, o, r = mixed

    def batch(seed):
        rr = np.random.default_rng(seed)
        return [(rr.integers(0, 48, 12).astype(np.uint32), 5) for _ in range(10)]
    q1, q2 = batch(6), batch(7)
    off, ln, pool = thr.thr_query_batch(g, q1)
    _check(g, o, q1, off, ln, pool)
    off, ln, pool = thr.thr_query_batch(g, q2)
    assert thr.thr_last_batch_info()["graph"] == 1
    _check(g, o, q2, off, ln, pool)


def test_identical_plans_relaunch_the_cached_graph(mixed):
    """Batches of one shape into the same device pool, alternating two id sets
    (A, B, A, B): when every parameter of the captured work is unchanged the
    cached executable is launched as it is, reading the new plan from the
    pinned staging; each result is that of its own queries."""
    import torch
    g, o, r = mixed
    rr = np.random.default_rng(17)
    qa = [(rr.integers(0, 48, 12).astype(np.uint32), 4) for _ in range(6)]
    qb = [(rr.integers(0, 48, 12).astype(np.uint32), 4) for _ in range(6)]
    pool = torch.zeros(6 * (g.nwords + 1), dtype=torch.int64, device="cuda")
    for qs in (qa, qb, qa, qb):
        off, ln, _ = thr.thr_query_batch(g, qs, pool=pool)
        host = pool.cpu().numpy().view(np.uint64)
        for k, (ids, T) in enumerate(qs):
            assert np.array_equal(host[int(off[k]): int(off[k] + ln[k])], o.threshold(ids, T))
    assert thr.thr_last_batch_info()["graph"] == 1


def test_relaunch_never_reuses_another_index():
    """Two indexes of the same shape queried alternately with batches of the
    same shape into the same device pool, then one freed and a new one built
    in its place: every result is that of the index it was asked of."""
    import torch
    r = 3 * 8192 + 1000
    pairs = []
    for seed in (41, 42, 43):
        arrays = [synth.bernoulli(seed, i, r, 0.05 + 0.02 * i) for i in range(12)]
        gw, goff = thr.encode_many(arrays, r)
        pairs.append((thr.idx_build_rle(gw, goff, r),
                      oracle.Index([oracle.encode(a, r) for a in arrays], r)))
    qs = [(np.arange(12, dtype=np.uint32), T) for T in (2, 3)]
    pool = torch.zeros(2 * (pairs[0][0].nwords + 1), dtype=torch.int64, device="cuda")

    def check(g, o):
        off, ln, _ = thr.thr_query_batch(g, qs, pool=pool)
        host = pool.cpu().numpy().view(np.uint64)
        for k, (ids, T) in enumerate(qs):
            assert np.array_equal(host[int(off[k]): int(off[k] + ln[k])], o.threshold(ids, T))
    for g, o in (pairs[0], pairs[1], pairs[0], pairs[1]):
        check(g, o)
    pairs[0][0].close()
    check(*pairs[2])
    check(*pairs[1])
    pairs[1][0].close()
    pairs[2][0].close()


def test_batch_many_inputs_per_query(mixed):
    """n above one chunk of input records (128) and above the 8-bit
    ScanCount counters (255): the uncached id path and the 16-bit counters."""
    g, o, r = mixed
    rng = np.random.default_rng(8)
    qs = [(rng.integers(0, 48, 300).astype(np.uint32), 140),
          (rng.integers(0, 48, 200).astype(np.uint32), 1),
          (rng.integers(0, 48, 129).astype(np.uint32), 129),
          (rng.integers(0, 48, 260).astype(np.uint32), 30)]
    for fl in (0, thr.THR_VARIANT_SCANCOUNT, thr.THR_VARIANT_POSITION, thr.THR_VARIANT_SPLIT,
               thr.THR_POLICY_RULE):
        off, ln, pool = thr.thr_query_batch(g, qs, flags=fl)
        _check(g, o, qs, off, ln, pool)


@pytest.mark.parametrize("flags", [thr.THR_VARIANT_SCANCOUNT, thr.THR_VARIANT_POSITION,
                                   thr.THR_VARIANT_SPLIT, thr.THR_POLICY_RULE,
                                   thr.THR_POLICY_LEARNED])
def test_batch_policies(mixed, flags):
    g, o, r = mixed
    qs = _queries(9, 48, 30)
    off, ln, pool = thr.thr_query_batch(g, qs, flags=flags)
    _check(g, o, qs, off, ln, pool)


def test_batch_pool_too_small(mixed):
    g, o, r = mixed
    qs = _queries(10, 48, 12)
    off, ln, pool = thr.thr_query_batch(g, qs)
    need = int(ln.sum())
    small = np.zeros(max(need - 1, 1), np.uint64)
    with pytest.raises(thr.ThrError) as e:
        thr.thr_query_batch(g, qs, pool=small)
    assert e.value.status == thr.THR_E_NOSPACE


def test_batch_many_criteria_full_size(many_criteria_full):
    """The 64 x 2^26 many-criteria bitmaps, the four thresholds as one batch
    (one counting pass shared by the four: same inputs) plus a query over
    other inputs (a second kernel class side by side), against the oracle."""
    arrays, r = many_criteria_full
    g, o = _index(arrays, r)
    ids = np.arange(synth.MANY_N, dtype=np.uint32)
    qs = [(ids, T) for T in synth.MANY_TS] + [(ids[:40], 2)]
    off, ln, pool = thr.thr_query_batch(g, qs)
    assert thr.thr_last_batch_info()["launches"] == 2
    _check(g, o, qs, off, ln, pool)
    off, ln, pool = thr.thr_query_batch(g, qs, flags=thr.THR_NO_GRAPH)
    _check(g, o, qs, off, ln, pool)


@pytest.mark.parametrize("cfg", range(16))
def test_every_launch_configuration(mixed, monkeypatch, cfg):
    """Work order, class merging, grid split and dynamic work fetch change
    only the schedule: every configuration gives the oracle's results."""
    g, o, r = mixed
    monkeypatch.setenv("THR_TUNE_CONFIG", str(cfg))
    qs = _queries(20 + cfg, 48, 24, nmax=300)
    off, ln, pool = thr.thr_query_batch(g, qs, flags=thr.THR_POLICY_RULE)
    assert thr.thr_last_batch_info()["config"] == cfg
    _check(g, o, qs, off, ln, pool)


def test_autotune_keeps_the_fastest(mixed):
    g, o, r = mixed
    qs = _queries(30, 48, 16)
    before = thr.thr_query_batch(g, qs)
    best, times = thr.thr_autotune(g, qs, reps=2)
    assert 0 <= best < 16 and len(times) == 16 and all(t > 0 for t in times)
    assert times[best] == min(times)
    off, ln, pool = thr.thr_query_batch(g, qs)
    assert thr.thr_last_batch_info()["config"] == best
    assert np.array_equal(ln, before[1])
    _check(g, o, qs, off, ln, pool)


def test_queries_sharing_inputs_count_once(mixed, monkeypatch):
    """Queries over the same id multiset (in any order, with repeats) share
    one counting pass: results per threshold equal the oracle's, every
    threshold kind included (0, 1, close to n, n, n + 1), and the group needs
    one pass-A launch."""
    g, o, r = mixed
    rng = np.random.default_rng(41)
    base = rng.integers(0, 48, 30).astype(np.uint32)
    qs = []
    for T in (0, 1, 2, 5, 15, 28, 29, 30, 31):
        qs.append((rng.permutation(base), T))
    other = rng.integers(0, 48, 12).astype(np.uint32)
    qs += [(other, 3), (np.concatenate([other, other[:2]]), 3)]  # not the same multiset
    off, ln, pool = thr.thr_query_batch(g, qs)
    _check(g, o, qs, off, ln, pool)
    # one launch counts the group (5-bit counters for T <= 30), one the rest
    assert thr.thr_last_batch_info()["launches"] <= 2
    # without sharing: the same results, every query counting for itself
    off2, ln2, pool2 = thr.thr_query_batch(g, qs, flags=thr.THR_NO_SHARE)
    assert np.array_equal(ln, ln2)
    assert np.array_equal(pool[: int(ln.sum())], pool2[: int(ln2.sum())])
    # groups never span chunks: with 4 slots per chunk the results still hold
    monkeypatch.setenv("THR_MAX_SLOTS", "4")
    off, ln, pool = thr.thr_query_batch(g, qs)
    _check(g, o, qs, off, ln, pool)
