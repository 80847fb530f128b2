"""Builders of the large synthetic indexes (serving and similarity
workloads) from the seeded generators of ``synth``.

The bitmaps are drawn as row lists and encoded with the library's row
encoder (thr_rle_encode_rows) in a spawned process pool, so that no
uncompressed bitmap of 2^26 rows is ever formed; the streams are then
concatenated and uploaded with idx_build_rle.

  serving     2^14 bitmaps over 2^26 rows, densities min(0.3, 0.3 k^-1.1),
              odd k i.i.d., even k clustered (runs of mean 256 rows)
  similarity  2^16 term bitmaps over 2^24 documents, densities
              min(0.3, C k^-1.1) summing to 110 (the mean document length),
              i.i.d.; 4096 queries of N ~ U[10, 200] Zipf-drawn terms with a
              prototype row planted in their N bitmaps, T = ceil(N / 2)
  sparse      i.i.d. Bernoulli(p) bitmaps (defaults 4096 over 2^24 rows,
              p = 2e-4), the inputs where ScanCount's per-set-bit cost pays
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402


def _encode_one(args):
    seed, k, r, p, clustered, planted = args
    import paper_1402_4466_gb300 as thr
    rows = synth.bitmap_rows(seed, k, r, p, clustered)
    if planted is not None and len(planted):
        rows = np.union1d(rows, np.asarray(planted, np.int64))
    return thr.thr_rle_encode_rows(rows, r)


def encode_family(jobs, workers: int = 0, chunk: int = 64):
    """Streams of the bitmaps described by jobs (seed, k, r, p, clustered,
    planted rows or None), in order; (words, offsets)."""
    if workers and workers > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=workers,
                                 mp_context=mp.get_context("spawn")) as ex:
            streams = list(ex.map(_encode_one, jobs, chunksize=chunk))
    else:
        streams = [_encode_one(j) for j in jobs]
    offsets = np.zeros(len(streams) + 1, np.uint64)
    offsets[1:] = np.cumsum([len(s) for s in streams])
    words = np.concatenate(streams) if streams else np.zeros(0, np.uint64)
    return words, offsets


def serving(nb: int = 1 << 14, r: int = 1 << 26, seed: int = 0, workers: int = 0):
    """(words, offsets, r) of the serving index."""
    dens = synth.serving_densities(nb)
    jobs = [(seed, k, r, float(dens[k - 1]), k % 2 == 0, None) for k in range(1, nb + 1)]
    words, offsets = encode_family(jobs, workers)
    return words, offsets, r


def similarity(nb: int = 1 << 16, r: int = 1 << 24, nq: int = 4096, seed: int = 0,
               workers: int = 0):
    """(words, offsets, r, queries, prototype rows) of the similarity index
    and its batch."""
    dens = synth.similarity_densities(nb)
    queries, planted, protos = synth.similarity_queries(seed, nq, dens, r)
    jobs = [(seed, k, r, float(dens[k]), False, planted.get(k)) for k in range(nb)]
    words, offsets = encode_family(jobs, workers)
    return words, offsets, r, queries, protos


def sparse(nb: int = 4096, r: int = 1 << 24, p: float = 2e-4, seed: int = 0, workers: int = 0):
    """(words, offsets) of nb i.i.d. Bernoulli(p) bitmaps over r rows (the
    very sparse inputs of the counting-variant comparison)."""
    jobs = [(seed, k, r, float(p), False, None) for k in range(nb)]
    return encode_family(jobs, workers)
