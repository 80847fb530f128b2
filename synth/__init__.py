"""Seeded synthetic bitmap generators shared by the tests, the oracle checks
and the benchmark.

This module only draws random bitmaps: it returns *uncompressed* 64-bit words
(bit j of word i is row 64*i + j, the least-significant bit being the smallest
row, Sec. 3.1 of Kaser & Lemire).  It holds none of the threshold method's
arithmetic and no stream encoder: each consumer encodes the words with its own
codec (the oracle with ``oracle.encode``, the GPU library with
``thr_rle_encode``).

Recipes (the paper's datasets are not available; these stand in for them):

* ``bernoulli``  -- every row set independently with probability p.  The set
  rows are the partial sums of Geometric(p) gaps (an exact Bernoulli process).
* ``clustered``  -- runs of ones with Geometric lengths of mean ``mean_run``
  alternating with Geometric gaps of mean ``mean_run*(1-p)/p``, starting with
  a gap, so that the expected density is p.
* ``many_criteria`` -- N bitmaps over r rows with densities log-uniform in
  [1e-4, 0.3]; the first half Bernoulli, the second half clustered.
* ``plain`` -- N Bernoulli(p) bitmaps of equal density.

Every generator is a pure function of its arguments (seed included).
"""
from __future__ import annotations

import math

import numpy as np


def nwords(r: int) -> int:
    return (int(r) + 63) // 64


def _rng(seed: int, *stream: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), *map(int, stream)]))


def rows_to_words(rows: np.ndarray, r: int) -> np.ndarray:
    """Pack sorted or unsorted row numbers (< r) into uncompressed words."""
    W = nwords(r)
    bits = np.zeros(W * 64, dtype=np.bool_)
    if len(rows):
        bits[np.asarray(rows, dtype=np.int64)] = True
    return np.packbits(bits, bitorder="little").view("<u8").astype(np.uint64)


def runs_to_words(starts: np.ndarray, lengths: np.ndarray, r: int) -> np.ndarray:
    """Uncompressed words of the union of row intervals [start, start+len)."""
    W = nwords(r)
    edge = np.zeros(W * 64 + 1, dtype=np.int32)
    s = np.asarray(starts, dtype=np.int64)
    e = np.minimum(s + np.asarray(lengths, dtype=np.int64), r)
    keep = s < r
    np.add.at(edge, s[keep], 1)
    np.add.at(edge, e[keep], -1)
    bits = np.cumsum(edge[:-1]) > 0
    return np.packbits(bits, bitorder="little").view("<u8").astype(np.uint64)


def words_to_bits(words: np.ndarray, r: int) -> np.ndarray:
    """Boolean row vector of an uncompressed bitmap (helper for tests)."""
    w = np.ascontiguousarray(words, dtype=np.uint64)
    return np.unpackbits(w.view(np.uint8), bitorder="little")[: int(r)].astype(bool)


def bernoulli_rows(rng: np.random.Generator, r: int, p: float) -> np.ndarray:
    """Set rows of an i.i.d. Bernoulli(p) bitmap over r rows."""
    if p <= 0 or r == 0:
        return np.zeros(0, dtype=np.int64)
    if p >= 1:
        return np.arange(r, dtype=np.int64)
    if p > 0.5:  # draw the zeros instead and complement
        zeros = bernoulli_rows(rng, r, 1.0 - p)
        keep = np.ones(r, dtype=np.bool_)
        keep[zeros] = False
        return np.nonzero(keep)[0]
    out = []
    pos = -1
    expect = r * p
    while True:
        k = int(expect + 6 * math.sqrt(expect + 1) + 64)
        gaps = rng.geometric(p, size=k).astype(np.int64)
        cand = pos + np.cumsum(gaps)
        inside = cand[cand < r]
        out.append(inside)
        if len(inside) < len(cand):
            break
        pos = int(cand[-1])
        expect = (r - pos) * p
    return np.concatenate(out)


def bernoulli(seed: int, k: int, r: int, p: float) -> np.ndarray:
    return rows_to_words(bernoulli_rows(_rng(seed, 1, k), r, p), r)


def clustered(seed: int, k: int, r: int, p: float, mean_run: float = 256.0) -> np.ndarray:
    """Runs of ones (Geometric, mean mean_run) between Geometric gaps of mean
    mean_run*(1-p)/p, starting with a gap."""
    rng = _rng(seed, 2, k)
    if p <= 0 or r == 0:
        return np.zeros(nwords(r), dtype=np.uint64)
    mean_gap = max(mean_run * (1.0 - p) / p, 1.0)
    starts, lens = [], []
    pos = 0
    while pos < r:
        ncyc = int((r - pos) / (mean_run + mean_gap) * 1.2) + 16
        gaps = rng.geometric(1.0 / mean_gap, size=ncyc).astype(np.int64)
        runs = rng.geometric(1.0 / mean_run, size=ncyc).astype(np.int64)
        cyc = gaps + runs
        ends = pos + np.cumsum(cyc)
        st = ends - runs
        starts.append(st)
        lens.append(runs)
        pos = int(ends[-1])
    s = np.concatenate(starts)
    l = np.concatenate(lens)
    keep = s < r
    return runs_to_words(s[keep], l[keep], r)


def log_uniform_densities(seed: int, n: int, lo: float = 1e-4, hi: float = 0.3) -> np.ndarray:
    rng = _rng(seed, 3)
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))


def _many_one(args):
    seed, k, r, p, clustered_kind = args
    return clustered(seed, k, r, p) if clustered_kind else bernoulli(seed, k, r, p)


def many_criteria(seed: int, n: int, r: int, lo: float = 1e-4, hi: float = 0.3,
                  workers: int = 0):
    """N bitmaps, densities log-uniform in [lo, hi]; first half Bernoulli,
    second half clustered (mean run 256 rows).  Returns (words list, densities).
    workers > 1 draws the bitmaps in a spawned process pool (same result)."""
    dens = log_uniform_densities(seed, n, lo, hi)
    half = n // 2
    jobs = [(seed, k, r, float(dens[k]), k >= half) for k in range(n)]
    if workers and workers > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(max_workers=workers,
                                 mp_context=mp.get_context("spawn")) as ex:
            out = list(ex.map(_many_one, jobs))
    else:
        out = [_many_one(j) for j in jobs]
    return out, dens


def plain(seed: int, n: int, r: int, p: float):
    """N i.i.d. Bernoulli(p) bitmaps over r rows."""
    return [bernoulli(seed, k, r, p) for k in range(n)]


# The two workloads run end to end on one GPU (sizes named, not numbered).
PLAIN_N, PLAIN_R, PLAIN_P, PLAIN_T = 8, 1 << 20, 0.05, 4
MANY_N, MANY_R, MANY_TS = 64, 1 << 26, (2, 16, 32, 63)
