"""Row-range sharding on the CPU: slicing canonical streams into 64-row-
aligned shards and stitching shard results back (thr_rle_slice /
thr_rle_stitch), checked against the oracle; and the multi-process path of
`sharded.ShardedIndex` with two gloo ranks whose shard results come from the
CPU oracle (no GPU), which must equal the oracle's result over all rows."""
import os
import socket

import numpy as np
import pytest

import oracle
import paper_1402_4466_gb300 as thr
import synth
from paper_1402_4466_gb300 import sharded


def _bitmaps(seed, n, r):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = i % 4
        if kind == 0:
            out.append(synth.bernoulli(seed, i, r, float(10 ** rng.uniform(-3, -0.3))))
        elif kind == 1:
            out.append(synth.clustered(seed, i, r, float(rng.uniform(0.05, 0.6))))
        elif kind == 2:  # long fills across shard seams
            rows = np.concatenate([np.arange(r // 3, 2 * r // 3), [r - 1]])
            out.append(synth.rows_to_words(rows, r))
        else:
            out.append(np.zeros(synth.nwords(r), np.uint64))
    return out


@pytest.mark.parametrize("r", [64, 65, 1000, 200_003, 70_000])
def test_slice_then_stitch_is_identity(r):
    arrays = _bitmaps(3, 8, r)
    W = synth.nwords(r)
    rng = np.random.default_rng(r)
    for a in arrays:
        s = oracle.encode(a, r)
        cuts = sorted(set(rng.integers(1, W, size=min(4, max(W - 1, 0))).tolist())) if W > 1 else []
        bounds = [0] + cuts + [W]
        parts, rows = [], []
        for w0, w1 in zip(bounds[:-1], bounds[1:]):
            p = thr.thr_rle_slice(s, r, w0, w1)
            nrows = min(64 * w1, r) - 64 * w0
            # each slice is the canonical stream of its own rows
            assert np.array_equal(p, oracle.encode(a[w0:w1], nrows))
            parts.append(p)
            rows.append(nrows)
        assert np.array_equal(thr.thr_rle_stitch(parts, rows), s)


def test_stitched_shard_results_equal_the_whole():
    r = 300_000 + 17
    arrays = _bitmaps(5, 12, r)
    streams = [oracle.encode(a, r) for a in arrays]
    words, offsets = oracle.concat(streams)
    whole = oracle.Index(streams, r)
    for world in (2, 3, 5):
        ranges = sharded.shard_ranges(r, world)
        assert sum(rows for _, rows in ranges) == r
        shards = []
        for row0, rows in ranges:
            sw, so = sharded.slice_index(words, offsets, r, row0, rows)
            shards.append((oracle.Index([sw[int(so[i]):int(so[i + 1])] for i in range(12)], rows),
                           rows))
        for ids, T in (([0, 1, 2, 3], 1), ([0, 1, 2, 3, 4, 5], 2), (list(range(12)), 4),
                       ([1, 1, 2, 5, 9], 3), (list(range(12)), 12), ([2, 6, 10], 3)):
            parts = [ix.threshold(ids, T) for ix, _ in shards]
            got = thr.thr_rle_stitch(parts, [rows for _, rows in shards])
            assert np.array_equal(got, whole.threshold(ids, T)), (world, ids, T)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _partial_hist(ix, ids, K):
    """A shard's answer and its count histogram as the GPU profiling pass
    gives them: exact for counts >= max(T, 1), bins below that (and bin 0)
    not computed (zero here)."""
    T, _ = ix.opt_threshold(ids, K)
    h = ix.count_histogram(ids).copy()
    h[: max(T, 1)] = 0
    return T, h


def test_opt_threshold_over_shards_combines_histograms():
    r = 200_000 + 3
    arrays = _bitmaps(11, 10, r)
    streams = [oracle.encode(a, r) for a in arrays]
    words, offsets = oracle.concat(streams)
    whole = oracle.Index(streams, r)
    for world in (2, 3, 5):
        shards = []
        for row0, rows in sharded.shard_ranges(r, world):
            sw, so = sharded.slice_index(words, offsets, r, row0, rows)
            shards.append((oracle.Index([sw[int(so[i]):int(so[i + 1])] for i in range(10)],
                                        rows), rows))
        for ids in ([0, 1, 2, 3], list(range(10)), [1, 1, 4, 8, 8], [3]):
            for K in (1, 7, 1000, r // 3, r, r + 1):
                got = [_partial_hist(ix, ids, K) for ix, _ in shards]
                T = sharded.combine_opt([h for _, h in got], [t for t, _ in got], K)
                Tw, want = whole.opt_threshold(ids, K)
                assert T == Tw, (world, ids, K)
                parts = [ix.threshold(ids, T) for ix, _ in shards]
                assert np.array_equal(thr.thr_rle_stitch(parts, [n for _, n in shards]), want)


def _rank_main(rank, world, port, r, seed, queries, out_dir, opt_queries=()):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    arrays = _bitmaps(seed, 10, r)
    streams = [oracle.encode(a, r) for a in arrays]
    words, offsets = oracle.concat(streams)
    row0, rows = sharded.shard_ranges(r, world)[rank]
    sw, so = sharded.slice_index(words, offsets, r, row0, rows)
    local = oracle.Index([sw[int(so[i]):int(so[i + 1])] for i in range(10)], rows)
    sh = sharded.ShardedIndex(words, offsets, r, rank, world,
                              local_query=lambda ids, T: local.threshold(ids, T),
                              build_index=False)
    results = [sh.query(ids, T) for ids, T in queries]
    for ids, K in opt_queries:
        T, res = sh.query_opt(ids, K, local_hist=lambda i, k: _partial_hist(local, i, k))
        results += [np.array([T], np.uint64), res]
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), *results)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_with_the_oracle(tmp_path):
    import torch.multiprocessing as mp
    r = 130_000 + 5
    queries = [([0, 1, 2, 3, 4], 2), (list(range(10)), 3), ([1, 1, 4, 8], 2), ([2, 6], 2)]
    opt_queries = [(list(range(10)), 1), ([0, 1, 2, 3, 4], 500), ([1, 1, 4, 8], 40_000)]
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, r, 7, queries, str(tmp_path), opt_queries),
                       nprocs=2, join=True, start_method="spawn")
    arrays = _bitmaps(7, 10, r)
    whole = oracle.Index([oracle.encode(a, r) for a in arrays], r)
    for rank in range(2):
        got = np.load(os.path.join(tmp_path, f"rank{rank}.npz"))
        for k, (ids, T) in enumerate(queries):
            assert np.array_equal(got[f"arr_{k}"], whole.threshold(ids, T))
        for j, (ids, K) in enumerate(opt_queries):
            T, want = whole.opt_threshold(ids, K)
            k = len(queries) + 2 * j
            assert int(got[f"arr_{k}"][0]) == T, (ids, K)
            assert np.array_equal(got[f"arr_{k + 1}"], want)
