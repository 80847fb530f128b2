"""Row-sharded threshold queries across processes (one per GPU).

The rows [0, r) are split into `world` consecutive ranges whose sizes are
multiples of 64 rows (the last takes the rest).  Rank g holds an index of
the slices of every bitmap over its range (thr_rle_slice), answers a query
on it, and the shard results are exchanged (torch.distributed all-gather of
the compressed streams) and stitched into the result over all rows
(thr_rle_stitch): the only exchange is the shards' results, and the stitch
touches O(1) words at each seam.

    sh = ShardedIndex(words, offsets, r, rank, world)   # builds the local index
    out = sh.query(ids, T)                              # on every rank
    T, out = sh.query_opt(ids, K)                       # opt-threshold over all rows

An opt-threshold query (the largest T whose result holds at least K rows)
over row shards needs one more exchange: each shard's profiling pass gives
its own answer T_g and its count histogram, exact at or above T_g
(thr_query_opt_hist); the histograms are summed and the largest T_g taken
across ranks (all-reduce), which fixes T for the whole (`combine_opt`), and
then every shard answers the threshold query at that T.

`ShardSet` runs every shard in one process (the same arithmetic, the
exchange replaced by lists): the way to test the sharded path on one GPU.
"""
from __future__ import annotations

import numpy as np

import paper_1402_4466_gb300 as thr


def shard_ranges(r: int, world: int):
    """(row0, rows) of each rank: 64-row-aligned, near-equal, last takes the rest."""
    W = (int(r) + 63) // 64
    per = W // world
    bounds = [min(W, k * per) for k in range(world)] + [W]
    out = []
    for k in range(world):
        w0, w1 = bounds[k], bounds[k + 1]
        row0 = 64 * w0
        rows = (min(64 * w1, int(r)) - row0) if k == world - 1 else 64 * (w1 - w0)
        out.append((row0, rows))
    return out


def slice_index(words, offsets, r: int, row0: int, rows: int):
    """(words, offsets) of every bitmap restricted to rows [row0, row0 + rows)."""
    w0 = row0 // 64
    w1 = w0 + (rows + 63) // 64
    parts = [thr.thr_rle_slice(words[int(offsets[i]):int(offsets[i + 1])], r, w0, w1)
             for i in range(len(offsets) - 1)]
    off = np.zeros(len(parts) + 1, np.uint64)
    off[1:] = np.cumsum([len(p) for p in parts])
    return np.concatenate(parts), off


def combine_opt(hists, Ts, K: int) -> int:
    """The opt-threshold answer for K over all shards, from each shard's
    answer T_g and count histogram (exact for counts >= max(T_g, 1)): the
    first c from n down to max(max_g T_g, 1) whose summed suffix reaches K,
    else 0.  The whole's answer is at least every T_g (a shard's K rows are
    rows of the whole), so only bins that every shard has exactly are read."""
    total = np.sum(np.stack([np.asarray(h, dtype=np.uint64) for h in hists]), axis=0)
    lo = max(max(int(t) for t in Ts), 1)
    suffix = 0
    for c in range(len(total) - 1, lo - 1, -1):
        suffix += int(total[c])
        if suffix >= K:
            return c
    return 0


class ShardSet:
    """Every row shard of an index in this process, on the current GPU:
    query() answers each shard and stitches the results, query_opt() combines
    the shards' histograms first (no collective: the exchange is a list)."""

    def __init__(self, words, offsets, r: int, shards: int):
        self.r = int(r)
        self.ranges = shard_ranges(r, shards)
        self.idx = []
        for row0, rows in self.ranges:
            w, o = slice_index(words, offsets, r, row0, rows)
            self.idx.append(thr.idx_build_rle(w, o, rows))

    def close(self):
        for g in self.idx:
            g.close()

    def query(self, ids, T: int) -> np.ndarray:
        parts = [thr.thr_query(g, ids, T) for g in self.idx]
        return thr.thr_rle_stitch(parts, [rows for _, rows in self.ranges])

    def query_opt(self, ids, K: int = 1):
        got = [thr.thr_query_opt_hist(g, ids, K) for g in self.idx]
        T = combine_opt([h for _, h in got], [t for t, _ in got], K)
        return T, self.query(ids, T)


class ShardedIndex:
    """The rank's shard of a row-sharded index.  `local_query(ids, T)` may
    replace the GPU query of the shard (it must return the shard's result
    stream); by default the shard lives on this rank's current GPU."""

    def __init__(self, words, offsets, r: int, rank: int, world: int, local_query=None,
                 build_index: bool = True):
        self.r, self.rank, self.world = int(r), rank, world
        self.ranges = shard_ranges(r, world)
        row0, rows = self.ranges[rank]
        self.words, self.offsets = slice_index(words, offsets, r, row0, rows)
        self.rows = rows
        self.idx = thr.idx_build_rle(self.words, self.offsets, rows) if build_index else None
        self.local_query = local_query or (lambda ids, T: thr.thr_query(self.idx, ids, T))

    def query_opt(self, ids, K: int = 1, group=None, local_hist=None):
        """(T, result) of the opt-threshold query over all rows: the shards'
        histograms summed (all-reduce) and their answers' maximum, combined
        by combine_opt, then the threshold query at T on every shard.
        local_hist(ids, K) -> (T_g, hist) may replace the shard's profiling
        pass (thr_query_opt_hist)."""
        import torch
        import torch.distributed as dist
        if local_hist is None:
            T_g, hist = thr.thr_query_opt_hist(self.idx, ids, K)
        else:
            T_g, hist = local_hist(ids, K)
        if self.world == 1:
            T = combine_opt([hist], [T_g], K)
        else:
            h = torch.from_numpy(np.asarray(hist, dtype=np.uint64).astype(np.int64))
            t = torch.tensor([int(T_g)], dtype=torch.int64)
            dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
            dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
            T = combine_opt([h.numpy().astype(np.uint64)], [int(t.item())], K)
        return T, self.query(ids, T, group=group)

    def query(self, ids, T: int, group=None) -> np.ndarray:
        import torch.distributed as dist
        mine = np.asarray(self.local_query(ids, T), dtype=np.uint64)
        if self.world == 1:
            return thr.thr_rle_stitch([mine], [self.rows])
        parts = [None] * self.world
        dist.all_gather_object(parts, mine, group=group)
        return thr.thr_rle_stitch(parts, [rows for _, rows in self.ranges])
