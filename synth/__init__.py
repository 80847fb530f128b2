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
* ``serving_densities`` -- Zipf(1.1) densities 0.3 k^-1.1 of the serving
  index (odd k i.i.d., even k clustered).
* ``similarity_densities`` / ``similarity_queries`` -- term densities
  min(0.3, C k^-1.1) summing to the mean document length, and queries of
  N ~ U[10, 200] Zipf-drawn terms with a planted prototype row, T = ceil(N/2).
* ``bitmap_rows`` -- the same bitmaps as row lists (for encoders that take
  rows, when the uncompressed words would be too large).

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


def clustered_runs(seed: int, k: int, r: int, p: float, mean_run: float = 256.0):
    """(starts, lengths) of the runs of ones of a clustered bitmap: Geometric
    run lengths of mean mean_run between Geometric gaps of mean
    mean_run*(1-p)/p, starting with a gap."""
    rng = _rng(seed, 2, k)
    if p <= 0 or r == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
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
    s, l = s[keep], l[keep]
    return s, np.minimum(l, r - s)


def clustered(seed: int, k: int, r: int, p: float, mean_run: float = 256.0) -> np.ndarray:
    """Uncompressed words of the clustered bitmap of ``clustered_runs``."""
    if p <= 0 or r == 0:
        return np.zeros(nwords(r), dtype=np.uint64)
    s, l = clustered_runs(seed, k, r, p, mean_run)
    return runs_to_words(s, l, r)


def runs_to_rows(starts: np.ndarray, lengths: np.ndarray) -> np.ndarray:
    """Ascending rows of disjoint ascending runs [start, start + length)."""
    if len(starts) == 0:
        return np.zeros(0, np.int64)
    lengths = np.asarray(lengths, np.int64)
    total = int(lengths.sum())
    base = np.repeat(np.asarray(starts, np.int64) - np.concatenate(([0], np.cumsum(lengths)[:-1])),
                     lengths)
    return base + np.arange(total, dtype=np.int64)


def bitmap_rows(seed: int, k: int, r: int, p: float, is_clustered: bool) -> np.ndarray:
    """Set rows (ascending) of bitmap k of a family: the same draws as
    ``bernoulli`` / ``clustered`` with these arguments."""
    if is_clustered:
        return runs_to_rows(*clustered_runs(seed, k, r, p))
    return bernoulli_rows(_rng(seed, 1, k), r, p)


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


def serving_densities(nb: int, scale: float = 0.3, s: float = 1.1) -> np.ndarray:
    """Densities of the serving workload: bitmap k (1-based) has
    min(0.3, scale * k^-s); odd k are i.i.d., even k clustered."""
    k = np.arange(1, nb + 1, dtype=np.float64)
    return np.minimum(0.3, scale * k ** -s)


def similarity_densities(nb: int, mean_len: float = 110.0, s: float = 1.1,
                         cap: float = 0.3) -> np.ndarray:
    """Term densities of the similarity workload: f_k = min(cap, C k^-s)
    with C chosen (bisection) so that the densities sum to the mean document
    length (a document of 20..200 terms, 110 on average)."""
    k = np.arange(1, nb + 1, dtype=np.float64)
    lo, hi = 0.0, 1e4
    for _ in range(200):
        C = 0.5 * (lo + hi)
        if np.minimum(cap, C * k ** -s).sum() < mean_len:
            lo = C
        else:
            hi = C
    return np.minimum(cap, 0.5 * (lo + hi) * k ** -s)


def similarity_queries(seed: int, nq: int, dens: np.ndarray, r: int, nmin: int = 10,
                       nmax: int = 200):
    """Queries of the similarity workload: N ~ U[nmin, nmax] distinct terms
    drawn with probability proportional to their density (Zipf weights), a
    prototype row (uniform) planted in those N bitmaps, T = ceil(N / 2).
    Returns (list of (ids, T), dict term -> planted rows, prototype row of
    every query)."""
    rng = _rng(seed, 7)
    w = dens / dens.sum()
    queries, planted, protos = [], {}, []
    for _ in range(nq):
        n = int(rng.integers(nmin, nmax + 1))
        ids = np.sort(rng.choice(len(dens), size=n, replace=False, p=w)).astype(np.uint32)
        row = int(rng.integers(0, r))
        for t in ids.tolist():
            planted.setdefault(t, []).append(row)
        queries.append((ids, (n + 1) // 2))
        protos.append(row)
    return queries, planted, protos


# The two workloads run end to end on one GPU (sizes named, not numbered).
PLAIN_N, PLAIN_R, PLAIN_P, PLAIN_T = 8, 1 << 20, 0.05, 4
MANY_N, MANY_R, MANY_TS = 64, 1 << 26, (2, 16, 32, 63)
