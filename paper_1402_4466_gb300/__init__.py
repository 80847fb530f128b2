"""Python binding of libthr: GPU threshold (T-overlap) queries over
run-length-compressed bitmaps (Kaser & Lemire, arXiv 1402.4466).

Argument marshalling only: every step of a query runs in the CUDA kernels of
``csrc/`` behind the C ABI of ``include/thr.h``.  The functions keep the ABI's
names.  There is no CPU fallback: if the library cannot be built or loaded,
``load()`` raises.

Arrays are numpy (host) or objects with ``data_ptr()`` and ``is_cuda``
(torch tensors, for device outputs); PyTorch is only used by callers for
device memory and streams.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

THR_OK, THR_E_INVAL, THR_E_FORMAT, THR_E_NOMEM = 0, 1, 2, 3
THR_E_NOSPACE, THR_E_CUDA, THR_E_TIMEOUT, THR_E_CHECK = 4, 5, 6, 7
THR_OUT_DEVICE = 0x1
THR_POLICY_PLAIN, THR_POLICY_RULE, THR_POLICY_LEARNED = 0x00, 0x10, 0x20
THR_POLICY_MASK = 0xF0
THR_PROFILE = 0x100
THR_NO_GRAPH = 0x1000
THR_NO_SHARE = 0x2000
THR_SYM_ODD = 0x4000
THR_VARIANT_CSA, THR_VARIANT_SCANCOUNT, THR_VARIANT_POSITION = 0x000, 0x200, 0x400
THR_VARIANT_SPLIT = 0x600
THR_VARIANT_LOOPED = 0x800
THR_VARIANT_STAGED = 0xA00
THR_MAX_IDS = 1048575  # bitmap ids (with repeats) per query: 2^20 - 1
THR_VARIANT_MASK = 0xE00

STATUS_NAMES = {0: "THR_OK", 1: "THR_E_INVAL", 2: "THR_E_FORMAT",
                3: "THR_E_NOMEM", 4: "THR_E_NOSPACE", 5: "THR_E_CUDA",
                6: "THR_E_TIMEOUT", 7: "THR_E_CHECK"}

# every symbol include/thr.h declares
ABI_SYMBOLS = ("idx_build_rle", "thr_query", "thr_query_batch", "thr_query_static", "idx_free",
               "thr_last_batch_info", "thr_autotune", "thr_select_variants", "thr_rule_model",
               "thr_selector_create", "thr_selector_free", "thr_selector_set_params",
               "thr_selector_get_params", "thr_selector_set_norm", "thr_selector_train",
               "thr_selector_predict", "thr_selector_gradients", "thr_query_features",
               "thr_index_set_selector", "thr_server_create", "thr_server_submit",
               "thr_server_wait", "thr_server_stats", "thr_server_free", "thr_rle_encode_rows",
               "thr_rle_slice", "thr_rle_stitch", "thr_query_sym", "thr_query_opt",
               "thr_query_opt_batch", "thr_query_opt_hist",
               "idx_info", "thr_rle_encode", "thr_rle_validate",
               "thr_last_kernel_ms", "thr_last_error")

_lock = threading.Lock()
_lib = None


class ThrError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


def checked() -> bool:
    """THR_CHECKED=1 in the environment selects the checked library
    (libthr_checked.so: bounds-checked query kernels, THR_E_CHECK)."""
    return os.environ.get("THR_CHECKED", "") == "1"


def library_path() -> str:
    return _build.LIB_CHECKED if checked() else _build.LIB


def load():
    """Build (when missing or stale) and load libthr.so (libthr_checked.so
    with THR_CHECKED=1); raises on failure."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(checked=checked())
            lib = ctypes.CDLL(path)
            u64, u32 = ctypes.c_uint64, ctypes.c_uint32
            vp, u64p, u32p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32)
            lib.idx_build_rle.argtypes = [vp, vp, u32, u64, vp, ctypes.POINTER(vp)]
            lib.thr_query.argtypes = [vp, vp, u32, u32, vp, u64, u64p, u32, vp]
            lib.thr_query_batch.argtypes = [vp, u32, vp, vp, vp, vp, u64, vp, vp, u32, vp]
            lib.thr_query_static.argtypes = [vp, vp, u32, u32, vp, u64, u64p, vp]
            lib.idx_free.argtypes = [vp]
            lib.idx_free.restype = None
            lib.idx_info.argtypes = [vp, u32p, u64p, u64p]
            lib.thr_rle_encode.argtypes = [vp, u64, u64, vp, u64, u64p]
            lib.thr_rle_validate.argtypes = [vp, u64, u64]
            lib.thr_rle_encode_rows.argtypes = [vp, u64, u64, vp, u64, u64p]
            lib.thr_rle_slice.argtypes = [vp, u64, u64, u64, u64, vp, u64, u64p]
            lib.thr_query_sym.argtypes = [vp, vp, u32, u32, u32, vp, u64, u64p, u32, vp]
            lib.thr_query_opt.argtypes = [vp, vp, u32, u64, u32p, vp, u64, u64p, u32, vp]
            lib.thr_query_opt_batch.argtypes = [vp, u32, vp, vp, vp, vp, vp, u64, vp, vp, u32,
                                                vp]
            lib.thr_query_opt_hist.argtypes = [vp, vp, u32, u64, u32p, vp, vp]
            lib.thr_rle_stitch.argtypes = [vp, vp, vp, u32, vp, u64, u64p]
            lib.thr_last_error.argtypes = []
            lib.thr_last_error.restype = ctypes.c_char_p
            lib.thr_last_kernel_ms.argtypes = []
            lib.thr_last_kernel_ms.restype = ctypes.c_double
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.thr_last_batch_info.argtypes = [u32p, u32p, i32p, u32p]
            lib.thr_autotune.argtypes = [vp, u32, vp, vp, vp, u32, u32, vp, vp, u32p]
            lib.thr_select_variants.argtypes = [vp, u32, vp, vp, vp, u32, vp]
            lib.thr_rule_model.argtypes = [vp, vp]
            lib.thr_selector_create.argtypes = [u64, u32, ctypes.POINTER(vp)]
            lib.thr_selector_free.argtypes = [vp]
            lib.thr_selector_free.restype = None
            lib.thr_selector_set_params.argtypes = [vp, vp]
            lib.thr_selector_get_params.argtypes = [vp, vp]
            lib.thr_selector_set_norm.argtypes = [vp, vp, vp]
            lib.thr_selector_train.argtypes = [vp, vp, vp, vp, u32, u32, u32, ctypes.c_float,
                                               u64, vp]
            lib.thr_selector_predict.argtypes = [vp, vp, u32, vp]
            lib.thr_selector_gradients.argtypes = [vp, vp, vp, vp, u32, vp, vp]
            lib.thr_query_features.argtypes = [vp, vp, u32, u32, vp]
            lib.thr_index_set_selector.argtypes = [vp, vp]
            lib.thr_server_create.argtypes = [vp, u32, u32, u64, u32, ctypes.POINTER(vp)]
            lib.thr_server_submit.argtypes = [vp, vp, u32, u32, u64p]
            lib.thr_server_wait.argtypes = [vp, u64, vp, u64, u64p,
                                            ctypes.POINTER(ctypes.c_double)]
            lib.thr_server_stats.argtypes = [vp, vp]
            lib.thr_server_free.argtypes = [vp]
            lib.thr_server_free.restype = None
            for f in ("idx_build_rle", "thr_query", "thr_query_batch", "thr_query_static", "idx_info",
                      "thr_rle_encode", "thr_rle_validate", "thr_last_batch_info",
                      "thr_autotune", "thr_select_variants", "thr_rule_model",
                      "thr_selector_create", "thr_selector_set_params", "thr_selector_get_params",
                      "thr_selector_set_norm", "thr_selector_train", "thr_selector_predict",
                      "thr_selector_gradients", "thr_query_features", "thr_index_set_selector",
                      "thr_server_create", "thr_server_submit", "thr_server_wait",
                      "thr_server_stats", "thr_rle_encode_rows", "thr_rle_slice",
                      "thr_rle_stitch", "thr_query_sym", "thr_query_opt_hist"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def thr_last_error() -> str:
    return load().thr_last_error().decode()


def thr_last_kernel_ms() -> float:
    return float(load().thr_last_kernel_ms())


def _check(st: int, where: str):
    if st != THR_OK:
        raise ThrError(st, where, thr_last_error())


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def _ptr(a) -> int:
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream(stream) -> int:
    if stream is None:
        return 0
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


class Index:
    """Handle of a device-resident index (idx_free on close / deletion)."""

    def __init__(self, handle: int, nbitmaps: int, r: int):
        self.handle = handle
        self.nbitmaps = nbitmaps
        self.r = r
        self.nwords = (r + 63) // 64

    def close(self):
        if self.handle:
            load().idx_free(ctypes.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        n = ctypes.c_uint32(0)
        r = ctypes.c_uint64(0)
        t = ctypes.c_uint64(0)
        _check(load().idx_info(ctypes.c_void_p(self.handle), ctypes.byref(n),
                               ctypes.byref(r), ctypes.byref(t)), "idx_info")
        return {"nbitmaps": n.value, "r": r.value, "total_words": t.value}


def idx_build_rle(words, offsets, r: int, stream=None) -> Index:
    """Device index from canonical streams concatenated in `words`, stream i
    being words[offsets[i]:offsets[i+1]]."""
    lib = load()
    w = _u64(words)
    o = _u64(offsets)
    h = ctypes.c_void_p(0)
    _check(lib.idx_build_rle(ctypes.c_void_p(w.ctypes.data if w.size else 0),
                             ctypes.c_void_p(o.ctypes.data), len(o) - 1, int(r),
                             ctypes.c_void_p(_stream(stream)), ctypes.byref(h)),
           "idx_build_rle")
    return Index(h.value, len(o) - 1, int(r))


def idx_free(idx: Index):
    idx.close()


def thr_query(idx: Index, ids, T: int, out=None, flags: int = 0, stream=None,
              cap: int | None = None):
    """Threshold query.  With out=None returns the result stream as a numpy
    array; with a device tensor `out` (THR_OUT_DEVICE is added) or a host
    array, fills it and returns the number of words written."""
    lib = load()
    ids = _u32(ids)
    n = ctypes.c_uint64(0)
    if out is None:
        buf = np.empty(idx.nwords + 1, dtype=np.uint64)
        _check(lib.thr_query(ctypes.c_void_p(idx.handle), ctypes.c_void_p(ids.ctypes.data),
                             ids.size, int(T), ctypes.c_void_p(buf.ctypes.data), buf.size,
                             ctypes.byref(n), int(flags), ctypes.c_void_p(_stream(stream))),
               "thr_query")
        return buf[: n.value].copy()
    if getattr(out, "is_cuda", False):
        flags |= THR_OUT_DEVICE
    size = cap if cap is not None else (out.numel() if hasattr(out, "numel") else out.size)
    st = lib.thr_query(ctypes.c_void_p(idx.handle), ctypes.c_void_p(ids.ctypes.data), ids.size,
                       int(T), ctypes.c_void_p(_ptr(out)), int(size), ctypes.byref(n),
                       int(flags), ctypes.c_void_p(_stream(stream)))
    if st == THR_E_NOSPACE:
        raise ThrError(st, "thr_query", f"needs {n.value} words")
    _check(st, "thr_query")
    return n.value


def thr_query_sym(idx: Index, ids, lo: int = 0, hi: int | None = None, odd: bool = False,
                  out=None, stream=None, flags: int = 0):
    """Rows whose count over ids lies in [lo, hi] (hi=None: n), or with
    odd=True whose count is odd.  Returns the stream (out=None) or fills a
    device tensor / host array and returns the number of words."""
    lib = load()
    ids = _u32(ids)
    hi = ids.size if hi is None else int(hi)
    flags |= THR_SYM_ODD if odd else 0
    n = ctypes.c_uint64(0)
    if out is None:
        buf = np.empty(idx.nwords + 1, dtype=np.uint64)
        _check(lib.thr_query_sym(ctypes.c_void_p(idx.handle), ctypes.c_void_p(ids.ctypes.data),
                                 ids.size, int(lo), hi, ctypes.c_void_p(buf.ctypes.data),
                                 buf.size, ctypes.byref(n), flags,
                                 ctypes.c_void_p(_stream(stream))), "thr_query_sym")
        return buf[: n.value].copy()
    if getattr(out, "is_cuda", False):
        flags |= THR_OUT_DEVICE
    size = out.numel() if hasattr(out, "numel") else out.size
    _check(lib.thr_query_sym(ctypes.c_void_p(idx.handle), ctypes.c_void_p(ids.ctypes.data),
                             ids.size, int(lo), hi, ctypes.c_void_p(_ptr(out)), int(size),
                             ctypes.byref(n), flags, ctypes.c_void_p(_stream(stream))),
           "thr_query_sym")
    return n.value


def thr_query_opt(idx: Index, ids, K: int = 1, out=None, stream=None, flags: int = 0):
    """Opt-threshold query: the largest T whose T-overlap result over ids
    holds at least K rows (0 when none does), and that result.  Returns
    (T, stream) with out=None, else fills a device tensor / host array and
    returns (T, number of words)."""
    lib = load()
    ids = _u32(ids)
    n = ctypes.c_uint64(0)
    T = ctypes.c_uint32(0)
    if out is None:
        buf = np.empty(idx.nwords + 1, dtype=np.uint64)
        _check(lib.thr_query_opt(ctypes.c_void_p(idx.handle), ctypes.c_void_p(ids.ctypes.data),
                                 ids.size, int(K), ctypes.byref(T),
                                 ctypes.c_void_p(buf.ctypes.data), buf.size, ctypes.byref(n),
                                 flags, ctypes.c_void_p(_stream(stream))), "thr_query_opt")
        return T.value, buf[: n.value].copy()
    if getattr(out, "is_cuda", False):
        flags |= THR_OUT_DEVICE
    size = out.numel() if hasattr(out, "numel") else out.size
    _check(lib.thr_query_opt(ctypes.c_void_p(idx.handle), ctypes.c_void_p(ids.ctypes.data),
                             ids.size, int(K), ctypes.byref(T), ctypes.c_void_p(_ptr(out)),
                             int(size), ctypes.byref(n), flags,
                             ctypes.c_void_p(_stream(stream))), "thr_query_opt")
    return T.value, n.value


def thr_query_opt_hist(idx: Index, ids, K: int = 1, stream=None):
    """The profiling pass of an opt-threshold query alone: (T, hist) with T
    this index's answer for K and hist[c] (c = 0..n) the rows counted exactly
    c times, exact for every c >= max(T, 1) (hist[0] is not computed)."""
    ids = _u32(ids)
    hist = np.zeros(ids.size + 1, dtype=np.uint64)
    T = ctypes.c_uint32(0)
    _check(load().thr_query_opt_hist(ctypes.c_void_p(idx.handle),
                                     ctypes.c_void_p(ids.ctypes.data), ids.size, int(K),
                                     ctypes.byref(T), ctypes.c_void_p(hist.ctypes.data),
                                     ctypes.c_void_p(_stream(stream))), "thr_query_opt_hist")
    return int(T.value), hist


def thr_query_opt_batch(idx: Index, queries, pool=None, flags: int = 0, stream=None):
    """Batch of (ids, K) opt-threshold queries.  Returns (T, out_off,
    out_len, pool); with pool=None a host pool of the worst-case size is
    allocated."""
    lib = load()
    nq, id_off, ids, _ = _pack([(q[0], 0) for q in queries])
    K = _u64([q[1] for q in queries])
    T = np.zeros(nq, dtype=np.uint32)
    if pool is None:
        pool = np.empty(max(nq * (idx.nwords + 1), 1), dtype=np.uint64)
    if getattr(pool, "is_cuda", False):
        flags |= THR_OUT_DEVICE
    size = pool.numel() if hasattr(pool, "numel") else pool.size
    out_off = np.zeros(nq, dtype=np.uint64)
    out_len = np.zeros(nq, dtype=np.uint64)
    _check(lib.thr_query_opt_batch(ctypes.c_void_p(idx.handle), nq,
                                   ctypes.c_void_p(id_off.ctypes.data),
                                   ctypes.c_void_p(ids.ctypes.data if ids.size else 0),
                                   ctypes.c_void_p(K.ctypes.data), ctypes.c_void_p(T.ctypes.data),
                                   ctypes.c_void_p(_ptr(pool)), int(size),
                                   ctypes.c_void_p(out_off.ctypes.data),
                                   ctypes.c_void_p(out_len.ctypes.data), int(flags),
                                   ctypes.c_void_p(_stream(stream))), "thr_query_opt_batch")
    return T, out_off, out_len, pool


def thr_query_raw(idx: Index, ids, T: int, out_ptr: int, cap: int, flags: int,
                  stream=None) -> tuple[int, int]:
    """ABI call with a raw output pointer; returns (status, out_len)."""
    ids = _u32(ids)
    n = ctypes.c_uint64(0)
    st = load().thr_query(ctypes.c_void_p(idx.handle), ctypes.c_void_p(ids.ctypes.data),
                          ids.size, int(T), ctypes.c_void_p(out_ptr), int(cap),
                          ctypes.byref(n), int(flags), ctypes.c_void_p(_stream(stream)))
    return st, n.value


def thr_query_static(idx: Index, ids, T: int, out, stream=None, cap: int | None = None) -> int:
    """thr_query_static: the query without any allocation (scratch in a fixed
    device array of the library); `out` must be device memory.  Returns the
    number of words written."""
    ids = _u32(ids)
    n = ctypes.c_uint64(0)
    size = cap if cap is not None else (out.numel() if hasattr(out, "numel") else out.size)
    st = load().thr_query_static(ctypes.c_void_p(idx.handle), ctypes.c_void_p(ids.ctypes.data),
                                 ids.size, int(T), ctypes.c_void_p(_ptr(out)), int(size),
                                 ctypes.byref(n), ctypes.c_void_p(_stream(stream)))
    if st == THR_E_NOSPACE:
        raise ThrError(st, "thr_query_static", f"needs {n.value} words")
    _check(st, "thr_query_static")
    return n.value


def thr_query_batch(idx: Index, queries, pool=None, flags: int = 0, stream=None):
    """Batch of (ids, T) queries.  Returns (out_off, out_len, pool); with
    pool=None a host pool of the worst-case size is allocated."""
    lib = load()
    nq, id_off, ids, T = _pack(queries)
    if pool is None:
        pool = np.empty(max(nq * (idx.nwords + 1), 1), dtype=np.uint64)
    if getattr(pool, "is_cuda", False):
        flags |= THR_OUT_DEVICE
    size = pool.numel() if hasattr(pool, "numel") else pool.size
    out_off = np.zeros(nq, dtype=np.uint64)
    out_len = np.zeros(nq, dtype=np.uint64)
    _check(lib.thr_query_batch(ctypes.c_void_p(idx.handle), nq,
                               ctypes.c_void_p(id_off.ctypes.data),
                               ctypes.c_void_p(ids.ctypes.data if ids.size else 0),
                               ctypes.c_void_p(T.ctypes.data), ctypes.c_void_p(_ptr(pool)),
                               int(size), ctypes.c_void_p(out_off.ctypes.data),
                               ctypes.c_void_p(out_len.ctypes.data), int(flags),
                               ctypes.c_void_p(_stream(stream))), "thr_query_batch")
    return out_off, out_len, pool


def thr_last_batch_info() -> dict:
    """Shape of this thread's last thr_query_batch call: chunks, pass-A
    launches, graph (1 cached graph replayed, 0 new graph, -1 no graph)."""
    c, l, g, k = ctypes.c_uint32(0), ctypes.c_uint32(0), ctypes.c_int32(0), ctypes.c_uint32(0)
    _check(load().thr_last_batch_info(ctypes.byref(c), ctypes.byref(l), ctypes.byref(g),
                                      ctypes.byref(k)), "thr_last_batch_info")
    return {"chunks": c.value, "launches": l.value, "graph": g.value, "config": k.value}


def _pack(queries):
    nq = len(queries)
    id_off = np.zeros(nq + 1, dtype=np.uint32)
    id_off[1:] = np.cumsum([len(q[0]) for q in queries])
    ids = _u32(np.concatenate([_u32(q[0]) for q in queries]) if nq else [])
    T = _u32([q[1] for q in queries])
    return nq, id_off, ids, T


def thr_autotune(idx: Index, queries, flags: int = 0, reps: int = 3, stream=None):
    """Time the 16 pass-A launch configurations on a sample batch of (ids, T)
    queries and keep the fastest for its shape in the index.  Returns
    (best configuration, list of median times in ms)."""
    nq, id_off, ids, T = _pack(queries)
    times = np.zeros(16, dtype=np.float64)
    best = ctypes.c_uint32(0)
    _check(load().thr_autotune(ctypes.c_void_p(idx.handle), nq,
                               ctypes.c_void_p(id_off.ctypes.data),
                               ctypes.c_void_p(ids.ctypes.data if ids.size else 0),
                               ctypes.c_void_p(T.ctypes.data), int(flags), int(reps),
                               ctypes.c_void_p(_stream(stream)),
                               ctypes.c_void_p(times.ctypes.data), ctypes.byref(best)),
           "thr_autotune")
    return best.value, times.tolist()


def thr_rle_encode(words, r: int) -> np.ndarray:
    """Canonical stream of uncompressed words (host codec of the library)."""
    lib = load()
    w = _u64(words)
    cap = w.size + 1
    out = np.empty(cap, dtype=np.uint64)
    n = ctypes.c_uint64(0)
    _check(lib.thr_rle_encode(ctypes.c_void_p(w.ctypes.data if w.size else 0), w.size, int(r),
                              ctypes.c_void_p(out.ctypes.data), cap, ctypes.byref(n)),
           "thr_rle_encode")
    return out[: n.value].copy()


def thr_rle_encode_rows(rows, r: int) -> np.ndarray:
    """Canonical stream of the bitmap with the given set rows (ascending)."""
    rows = np.ascontiguousarray(rows, dtype=np.uint64)
    cap = min(2 * rows.size + 2, (int(r) + 63) // 64 + 1)
    out = np.empty(max(cap, 1), dtype=np.uint64)
    n = ctypes.c_uint64(0)
    _check(load().thr_rle_encode_rows(ctypes.c_void_p(rows.ctypes.data if rows.size else 0),
                                      rows.size, int(r), ctypes.c_void_p(out.ctypes.data),
                                      out.size, ctypes.byref(n)), "thr_rle_encode_rows")
    return out[: n.value].copy()


def thr_rle_slice(stream, r: int, w0: int, w1: int) -> np.ndarray:
    """Canonical stream of the words [w0, w1) of a canonical stream."""
    s = _u64(stream)
    out = np.empty(min(2 * s.size + 2, w1 - w0 + 1), dtype=np.uint64)
    n = ctypes.c_uint64(0)
    _check(load().thr_rle_slice(ctypes.c_void_p(s.ctypes.data), s.size, int(r), int(w0), int(w1),
                                ctypes.c_void_p(out.ctypes.data), out.size, ctypes.byref(n)),
           "thr_rle_slice")
    return out[: n.value].copy()


def thr_rle_stitch(parts, rows) -> np.ndarray:
    """Canonical stream of consecutive row-range parts (rows[k] rows each)."""
    parts = [_u64(p) for p in parts]
    rows = np.ascontiguousarray(rows, dtype=np.uint64)
    ptrs = (ctypes.c_void_p * len(parts))(*[p.ctypes.data for p in parts])
    lens = np.array([p.size for p in parts], dtype=np.uint64)
    cap = int(sum(p.size for p in parts)) + 1
    out = np.empty(cap, dtype=np.uint64)
    n = ctypes.c_uint64(0)
    _check(load().thr_rle_stitch(ptrs, ctypes.c_void_p(lens.ctypes.data),
                                 ctypes.c_void_p(rows.ctypes.data), len(parts),
                                 ctypes.c_void_p(out.ctypes.data), out.size, ctypes.byref(n)),
           "thr_rle_stitch")
    return out[: n.value].copy()


def thr_rle_validate(stream, r: int) -> int:
    s = _u64(stream)
    return int(load().thr_rle_validate(ctypes.c_void_p(s.ctypes.data if s.size else 0),
                                       s.size, int(r)))


def encode_many(word_arrays, r: int):
    """Encode several uncompressed bitmaps; returns (concatenated words,
    offsets) ready for idx_build_rle."""
    streams = [thr_rle_encode(w, r) for w in word_arrays]
    offs = np.zeros(len(streams) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(s) for s in streams])
    return (np.concatenate(streams) if streams else np.zeros(0, np.uint64)), offs


# ------------------------------------------------------------------ selector

SEL_FEATURES, SEL_VARIANTS, SEL_PARAMS = 16, 4, 5508
THR_SEL_FP32 = 0x1
VARIANT_FLAGS = (THR_VARIANT_CSA, THR_VARIANT_POSITION, THR_VARIANT_SCANCOUNT,
                 THR_VARIANT_SPLIT)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


class Selector:
    """The learned cost model (thr_selector_*): 16 features -> 64 -> 64 -> 4
    predicted log pass-A times; BF16 weights (FP32 with fp32=True)."""

    def __init__(self, seed: int = 0, fp32: bool = False):
        h = ctypes.c_void_p(0)
        _check(load().thr_selector_create(int(seed), THR_SEL_FP32 if fp32 else 0,
                                          ctypes.byref(h)), "thr_selector_create")
        self.handle = h.value

    def close(self):
        if self.handle:
            load().thr_selector_free(ctypes.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(SEL_PARAMS, np.float32)
        _check(load().thr_selector_get_params(ctypes.c_void_p(self.handle),
                                              ctypes.c_void_p(out.ctypes.data)),
               "thr_selector_get_params")
        return out

    def set_params(self, p):
        p = _f32(p)
        assert p.size == SEL_PARAMS
        _check(load().thr_selector_set_params(ctypes.c_void_p(self.handle),
                                              ctypes.c_void_p(p.ctypes.data)),
               "thr_selector_set_params")

    def set_norm(self, mean, istd):
        mean, istd = _f32(mean), _f32(istd)
        _check(load().thr_selector_set_norm(ctypes.c_void_p(self.handle),
                                            ctypes.c_void_p(mean.ctypes.data),
                                            ctypes.c_void_p(istd.ctypes.data)),
               "thr_selector_set_norm")

    def train(self, X, T, M, epochs: int, batch: int = 512, lr: float = 1e-3,
              seed: int = 0) -> float:
        X, T = _f32(X), _f32(T)
        M = np.ascontiguousarray(M, dtype=np.uint8)
        loss = ctypes.c_float(0)
        _check(load().thr_selector_train(ctypes.c_void_p(self.handle),
                                         ctypes.c_void_p(X.ctypes.data),
                                         ctypes.c_void_p(T.ctypes.data),
                                         ctypes.c_void_p(M.ctypes.data), X.shape[0],
                                         int(epochs), int(batch), float(lr), int(seed),
                                         ctypes.byref(loss)), "thr_selector_train")
        return loss.value

    def predict(self, X) -> np.ndarray:
        X = _f32(X)
        Y = np.empty((X.shape[0], SEL_VARIANTS), np.float32)
        _check(load().thr_selector_predict(ctypes.c_void_p(self.handle),
                                           ctypes.c_void_p(X.ctypes.data), X.shape[0],
                                           ctypes.c_void_p(Y.ctypes.data)),
               "thr_selector_predict")
        return Y

    def gradients(self, X, T, M):
        X, T = _f32(X), _f32(T)
        M = np.ascontiguousarray(M, dtype=np.uint8)
        g = np.empty(SEL_PARAMS, np.float32)
        loss = ctypes.c_float(0)
        _check(load().thr_selector_gradients(ctypes.c_void_p(self.handle),
                                             ctypes.c_void_p(X.ctypes.data),
                                             ctypes.c_void_p(T.ctypes.data),
                                             ctypes.c_void_p(M.ctypes.data), X.shape[0],
                                             ctypes.c_void_p(g.ctypes.data), ctypes.byref(loss)),
               "thr_selector_gradients")
        return loss.value, g


def query_features(idx: Index, ids, T: int) -> np.ndarray:
    ids = _u32(ids)
    f = np.empty(SEL_FEATURES, np.float32)
    _check(load().thr_query_features(ctypes.c_void_p(idx.handle),
                                     ctypes.c_void_p(ids.ctypes.data), ids.size, int(T),
                                     ctypes.c_void_p(f.ctypes.data)), "thr_query_features")
    return f


def set_selector(idx: Index, sel: "Selector | None"):
    """Attach a cost model to the index (THR_POLICY_LEARNED uses it)."""
    _check(load().thr_index_set_selector(ctypes.c_void_p(idx.handle),
                                         ctypes.c_void_p(sel.handle if sel else 0)),
           "thr_index_set_selector")
    idx._selector = sel  # keep it alive while attached


def select_variants(idx: Index, queries, flags: int) -> np.ndarray:
    nq, id_off, ids, T = _pack(queries)
    out = np.zeros(max(nq, 1), np.uint8)
    _check(load().thr_select_variants(ctypes.c_void_p(idx.handle), nq,
                                      ctypes.c_void_p(id_off.ctypes.data),
                                      ctypes.c_void_p(ids.ctypes.data if ids.size else 0),
                                      ctypes.c_void_p(T.ctypes.data), int(flags),
                                      ctypes.c_void_p(out.ctypes.data)), "thr_select_variants")
    return out[:nq]


def rule_model(coeffs=None) -> np.ndarray:
    """Get (and with coeffs, first set) the rule chooser's 12 coefficients."""
    get = np.zeros(12, np.float64)
    setp = None
    if coeffs is not None:
        setp = np.ascontiguousarray(coeffs, dtype=np.float64)
        assert setp.size == 12
    _check(load().thr_rule_model(ctypes.c_void_p(setp.ctypes.data if setp is not None else 0),
                                 ctypes.c_void_p(get.ctypes.data)), "thr_rule_model")
    return get


# ------------------------------------------------------------------ serving

SERVER_STATS = ("done", "batches", "batched_queries", "max_in_flight", "max_batch",
                "max_claimed_bytes", "waiting", "in_flight")


class Server:
    """thr_server_*: continuous batching over a resident index.  submit()
    returns a ticket at once; wait(ticket) blocks for the result stream and
    its latency (ms, submit to completion)."""

    def __init__(self, idx: Index, workers: int = 4, max_batch: int = 64,
                 mem_budget: int = 4 << 30, flags: int = 0):
        h = ctypes.c_void_p(0)
        _check(load().thr_server_create(ctypes.c_void_p(idx.handle), int(workers),
                                        int(max_batch), int(mem_budget), int(flags),
                                        ctypes.byref(h)), "thr_server_create")
        self.handle = h.value
        self.idx = idx
        self._buf = np.empty(idx.nwords + 1, np.uint64)

    def submit(self, ids, T: int) -> int:
        ids = _u32(ids)
        t = ctypes.c_uint64(0)
        _check(load().thr_server_submit(ctypes.c_void_p(self.handle),
                                        ctypes.c_void_p(ids.ctypes.data), ids.size, int(T),
                                        ctypes.byref(t)), "thr_server_submit")
        return t.value

    def wait(self, ticket: int, buf: np.ndarray | None = None):
        buf = self._buf if buf is None else buf
        n = ctypes.c_uint64(0)
        lat = ctypes.c_double(0)
        _check(load().thr_server_wait(ctypes.c_void_p(self.handle), int(ticket),
                                      ctypes.c_void_p(buf.ctypes.data), buf.size,
                                      ctypes.byref(n), ctypes.byref(lat)), "thr_server_wait")
        return buf[: n.value].copy(), lat.value

    def stats(self) -> dict:
        a = np.zeros(8, np.uint64)
        _check(load().thr_server_stats(ctypes.c_void_p(self.handle),
                                       ctypes.c_void_p(a.ctypes.data)), "thr_server_stats")
        return {k: int(v) for k, v in zip(SERVER_STATS, a)}

    def close(self):
        if self.handle:
            load().thr_server_free(ctypes.c_void_p(self.handle))
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
