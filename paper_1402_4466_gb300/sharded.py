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

    def query(self, ids, T: int, group=None) -> np.ndarray:
        import torch.distributed as dist
        mine = np.asarray(self.local_query(ids, T), dtype=np.uint64)
        if self.world == 1:
            return thr.thr_rle_stitch([mine], [self.rows])
        parts = [None] * self.world
        dist.all_gather_object(parts, mine, group=group)
        return thr.thr_rle_stitch(parts, [rows for _, rows in self.ranges])
