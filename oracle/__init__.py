"""CPU oracle for the threshold (T-overlap) query over RLE-compressed bitmaps.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The GPU library (``paper_1402_4466_gb300``) neither imports it nor
shares any code with it.

The arithmetic lives in ``oracle.c`` (plain C, single-threaded): its own
stream decoder/validator, a ScanCount over decoded row lists (Sec. 5.1 of
Kaser & Lemire, arXiv 1402.4466) and its own canonical encoder.  This module
only compiles that file with gcc (on first use, or from ``build()``) and
marshals numpy arrays through ctypes.  ctypes releases the GIL during each
call, so independent queries may run on several host threads.

Parity status: every function is pinned by ``tests/test_oracle_pins.py`` (the
paper's worked examples, brute force on tiny inputs, independent Looped and
BSTM implementations, closed-form invariants and hand-written format cases);
``tests/test_oracle_mutants.py`` shows that plausible mistakes fail them.
The symmetric-function queries are pinned by ``tests/test_oracle_symmetric.py``
and the opt-threshold query by ``tests/test_oracle_opt.py`` (brute force, the
descending search of Sec. 5.2, the Looped route of Sec. 6.2, planted
mistakes).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_default = None

OK, E_INVAL, E_FORMAT, E_NOMEM, E_NOSPACE = 0, 1, 2, 3, 4


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def compile_c(src: str, out: str) -> str:
    """gcc -O2 -shared; plain C11, no machine-specific flags.  With OpenMP
    when the compiler has it (the row-partitioned ScanCount then runs its
    ranges on several threads), else without (they run one after another)."""
    tmp = out + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall", "-Wextra"]
    r = subprocess.run(base + ["-fopenmp", "-o", tmp, src], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base + ["-o", tmp, src], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (only when missing or stale)."""
    with _lock:
        if (force or not os.path.exists(_SO)
                or os.path.getmtime(_SO) < os.path.getmtime(SRC)):
            compile_c(SRC, _SO)
    return _SO


def nwords(r: int) -> int:
    return (int(r) + 63) // 64


def _p64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _p32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


class Oracle:
    """ctypes view of one compiled copy of oracle.c."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64, u32 = ctypes.c_uint64, ctypes.c_uint32
        lib.orc_encode.argtypes = [u64p, u64, u64, u64p, u64, u64p]
        lib.orc_decode.argtypes = [u64p, u64, u64, u64p, u64, u64p]
        lib.orc_validate.argtypes = [u64p, u64, u64]
        lib.orc_threshold.argtypes = [u64p, u64p, u32, u64, u32p, u32, u32,
                                      u64p, u64, u64p]
        lib.orc_threshold_words.argtypes = [u64p, u64p, u32, u64, u32p, u32,
                                            u32, u64p]
        lib.orc_symmetric.argtypes = [u64p, u64p, u32, u64, u32p, u32, u32, u32,
                                      ctypes.c_int, u64p, u64, u64p]
        lib.orc_opt_threshold.argtypes = [u64p, u64p, u32, u64, u32p, u32, u64, u32p,
                                          u64p, u64, u64p]
        lib.orc_threshold_parts.argtypes = [u64p, u64p, u32, u64, u32p, u32, u32, u32,
                                            u64p, u64, u64p]
        lib.orc_max_threads.argtypes = []
        lib.orc_count_histogram.argtypes = [u64p, u64p, u32, u64, u32p, u32, u64p]
        for f in (lib.orc_encode, lib.orc_decode, lib.orc_validate,
                  lib.orc_threshold, lib.orc_threshold_words, lib.orc_symmetric,
                  lib.orc_opt_threshold, lib.orc_threshold_parts, lib.orc_max_threads,
                  lib.orc_count_histogram):
            f.restype = ctypes.c_int
        self.c = lib

    def encode(self, words: np.ndarray, r: int) -> np.ndarray:
        """Canonical stream of the uncompressed words of an r-row bitmap."""
        w = np.ascontiguousarray(words, dtype=np.uint64)
        cap = w.size + 1
        out = np.empty(cap, dtype=np.uint64)
        n = ctypes.c_uint64(0)
        rc = self.c.orc_encode(_p64(w), w.size, int(r), _p64(out), cap,
                               ctypes.byref(n))
        if rc != OK:
            raise OracleError(rc, "encode")
        return out[: n.value].copy()

    def decode(self, stream: np.ndarray, r: int) -> np.ndarray:
        """Sorted set rows of a canonical stream (raises on a malformed one)."""
        s = np.ascontiguousarray(stream, dtype=np.uint64)
        rows = np.empty(max(int(r), 1), dtype=np.uint64)
        n = ctypes.c_uint64(0)
        rc = self.c.orc_decode(_p64(s), s.size, int(r), _p64(rows),
                               rows.size, ctypes.byref(n))
        if rc != OK:
            raise OracleError(rc, "decode")
        return rows[: n.value].copy()

    def validate(self, stream: np.ndarray, r: int) -> int:
        """0 when the stream is canonical for r rows, else an oracle status."""
        s = np.ascontiguousarray(stream, dtype=np.uint64)
        return int(self.c.orc_validate(_p64(s), s.size, int(r)))

    def threshold(self, words, offsets, r: int, ids, T: int) -> np.ndarray:
        """Canonical stream of the rows set in at least T of bitmaps ids."""
        words = np.ascontiguousarray(words, dtype=np.uint64)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        cap = nwords(r) + 1
        out = np.empty(cap, dtype=np.uint64)
        n = ctypes.c_uint64(0)
        rc = self.c.orc_threshold(_p64(words), _p64(offsets),
                                  len(offsets) - 1, int(r), _p32(ids),
                                  ids.size, int(T), _p64(out), cap,
                                  ctypes.byref(n))
        if rc != OK:
            raise OracleError(rc, "threshold")
        return out[: n.value].copy()

    def count_histogram(self, words, offsets, r: int, ids) -> np.ndarray:
        """hist[c], c = 0..n: the rows counted exactly c times over ids."""
        words = np.ascontiguousarray(words, dtype=np.uint64)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        hist = np.zeros(ids.size + 1, dtype=np.uint64)
        rc = self.c.orc_count_histogram(_p64(words), _p64(offsets), len(offsets) - 1, int(r),
                                        _p32(ids), ids.size, _p64(hist))
        if rc != OK:
            raise OracleError(rc, "count_histogram")
        return hist

    def max_threads(self) -> int:
        """Threads the row-partitioned query may use (1 without OpenMP)."""
        return int(self.c.orc_max_threads())

    def threshold_parts(self, words, offsets, r: int, ids, T: int,
                        parts: int) -> np.ndarray:
        """The threshold query with the rows cut into `parts` word ranges,
        each counted on its own (on OpenMP threads when available)."""
        words = np.ascontiguousarray(words, dtype=np.uint64)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        cap = nwords(r) + 1
        out = np.empty(cap, dtype=np.uint64)
        n = ctypes.c_uint64(0)
        rc = self.c.orc_threshold_parts(_p64(words), _p64(offsets), len(offsets) - 1, int(r),
                                        _p32(ids), ids.size, int(T), int(parts), _p64(out),
                                        cap, ctypes.byref(n))
        if rc != OK:
            raise OracleError(rc, "threshold_parts")
        return out[: n.value].copy()

    def symmetric(self, words, offsets, r: int, ids, lo: int, hi: int,
                  odd: bool = False) -> np.ndarray:
        """Canonical stream of the rows whose count c over ids satisfies
        lo <= c <= hi (or, with odd, whose c is odd)."""
        words = np.ascontiguousarray(words, dtype=np.uint64)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        cap = nwords(r) + 1
        out = np.empty(cap, dtype=np.uint64)
        n = ctypes.c_uint64(0)
        rc = self.c.orc_symmetric(_p64(words), _p64(offsets), len(offsets) - 1, int(r),
                                  _p32(ids), ids.size, int(lo), int(hi), 1 if odd else 0,
                                  _p64(out), cap, ctypes.byref(n))
        if rc != OK:
            raise OracleError(rc, "symmetric")
        return out[: n.value].copy()

    def opt_threshold(self, words, offsets, r: int, ids, K: int = 1):
        """(T, stream): the largest T whose T-overlap result over ids holds at
        least K rows (0 when none does), and that result."""
        words = np.ascontiguousarray(words, dtype=np.uint64)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        cap = nwords(r) + 1
        out = np.empty(cap, dtype=np.uint64)
        n = ctypes.c_uint64(0)
        T = ctypes.c_uint32(0)
        rc = self.c.orc_opt_threshold(_p64(words), _p64(offsets), len(offsets) - 1, int(r),
                                      _p32(ids), ids.size, int(K), ctypes.byref(T), _p64(out),
                                      cap, ctypes.byref(n))
        if rc != OK:
            raise OracleError(rc, "opt_threshold")
        return int(T.value), out[: n.value].copy()

    def threshold_words(self, words, offsets, r: int, ids, T: int) -> np.ndarray:
        """Uncompressed result words of the same query."""
        words = np.ascontiguousarray(words, dtype=np.uint64)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        out = np.zeros(max(nwords(r), 1), dtype=np.uint64)
        rc = self.c.orc_threshold_words(_p64(words), _p64(offsets),
                                        len(offsets) - 1, int(r), _p32(ids),
                                        ids.size, int(T), _p64(out))
        if rc != OK:
            raise OracleError(rc, "threshold_words")
        return out[: nwords(r)]


def load(path: str | None = None) -> Oracle:
    """The default oracle, or another compiled copy of oracle.c at path."""
    global _default
    if path is not None:
        return Oracle(path)
    if _default is None:
        build()
        _default = Oracle(_SO)
    return _default


def encode(words, r):
    return load().encode(words, r)


def decode(stream, r):
    return load().decode(stream, r)


def validate(stream, r):
    return load().validate(stream, r)


def concat(streams):
    """Concatenate streams; returns (words, offsets[n+1])."""
    streams = [np.asarray(s, dtype=np.uint64) for s in streams]
    offs = np.zeros(len(streams) + 1, dtype=np.uint64)
    if streams:
        offs[1:] = np.cumsum([len(s) for s in streams], dtype=np.uint64)
    cat = np.concatenate(streams) if streams else np.zeros(0, np.uint64)
    return np.ascontiguousarray(cat, dtype=np.uint64), offs


class Index:
    """Host-side set of streams (concatenated) that the oracle queries."""

    def __init__(self, streams, r: int, lib: Oracle | None = None):
        self.r = int(r)
        self.words, self.offsets = concat(list(streams))
        self.nbitmaps = len(self.offsets) - 1
        self.lib = lib

    def _o(self) -> Oracle:
        return self.lib if self.lib is not None else load()

    def stream(self, b: int) -> np.ndarray:
        return self.words[int(self.offsets[b]): int(self.offsets[b + 1])]

    def threshold(self, ids, T: int) -> np.ndarray:
        return self._o().threshold(self.words, self.offsets, self.r, ids, T)

    def threshold_words(self, ids, T: int) -> np.ndarray:
        return self._o().threshold_words(self.words, self.offsets, self.r,
                                         ids, T)

    def count_histogram(self, ids) -> np.ndarray:
        return self._o().count_histogram(self.words, self.offsets, self.r, ids)

    def threshold_parts(self, ids, T: int, parts: int) -> np.ndarray:
        return self._o().threshold_parts(self.words, self.offsets, self.r, ids, T, parts)

    def symmetric(self, ids, lo: int, hi: int, odd: bool = False) -> np.ndarray:
        return self._o().symmetric(self.words, self.offsets, self.r, ids, lo, hi, odd)

    def opt_threshold(self, ids, K: int = 1):
        return self._o().opt_threshold(self.words, self.offsets, self.r, ids, K)
