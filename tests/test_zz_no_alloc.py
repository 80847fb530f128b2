"""thr_query_static, the allocation-free query, against the CPU oracle and the
regular thr_query.

Some callers cannot allocate device memory while answering a query (their
GPU memory belongs to another allocator that reserved it up front, or they
must not risk an allocation failure or the synchronisation an allocation can
cause mid-work); thr_query_static keeps all of its scratch in one fixed
device array of the library.  Two calls in a row must each return exactly
what the oracle and thr_query return (the arithmetic is exact, so the
tolerance is zero); the largest accepted size (r = 2^26 rows) must run, and
sizes beyond the array's limits must be rejected.  This file runs last
(pytest collects it last) and also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle
import paper_1402_4466_gb300 as thr
import synth

pytestmark = pytest.mark.gpu


def _check(idx, oidx, queries):
    import torch
    outs = [torch.zeros(idx.nwords + 1, dtype=torch.int64, device="cuda") for _ in queries]
    lens = [thr.thr_query_static(idx, ids, T, out) for (ids, T), out in zip(queries, outs)]
    for (ids, T), out, n in zip(queries, outs, lens):
        want = oidx.threshold(ids, T)
        got = out[:n].cpu().numpy().view(np.uint64)
        assert n == len(want)
        assert np.array_equal(got, want)
        assert np.array_equal(thr.thr_query(idx, ids, T), want)


def test_static_scratch_query_matches_oracle():
    import torch
    assert torch.cuda.is_available()
    r = (1 << 20) + 77
    words, _ = synth.many_criteria(21, 24, r)
    gw, goff = thr.encode_many(words, r)
    idx = thr.idx_build_rle(gw, goff, r)
    oidx = oracle.Index([oracle.encode(w, r) for w in words], r)
    rng = np.random.default_rng(21)
    _check(idx, oidx, [(list(range(24)), 2), (rng.integers(0, 24, size=40).tolist(), 7)])
    idx.close()


def test_static_scratch_query_largest_accepted_size():
    # r = 2^26 rows is ceil(r/64) = 2^20 words, the largest the static
    # scratch takes: a few sparse bitmaps and an empty one
    import torch
    assert torch.cuda.is_available()
    r = 1 << 26
    words = [synth.bernoulli(5, k, r, p) for k, p in enumerate((1e-4, 3e-4, 1e-3))]
    words.append(np.zeros(synth.nwords(r), dtype=np.uint64))
    gw, goff = thr.encode_many(words, r)
    idx = thr.idx_build_rle(gw, goff, r)
    oidx = oracle.Index([oracle.encode(w, r) for w in words], r)
    _check(idx, oidx, [([0, 1, 2, 3], 1), ([0, 1, 2, 3, 2], 2)])
    idx.close()


def test_static_scratch_query_rejects_oversize():
    import torch
    r = (1 << 26) + 64  # one word more than the static scratch holds
    words = [np.zeros(synth.nwords(r), dtype=np.uint64)]
    gw, goff = thr.encode_many(words, r)
    idx = thr.idx_build_rle(gw, goff, r)
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(thr.ThrError) as e:
        thr.thr_query_static(idx, [0], 1, out)
    assert e.value.status == thr.THR_E_INVAL
    idx.close()
