"""thr_query_static, the allocation-free query, against the regular thr_query.

Some callers cannot allocate device memory while answering a query (their
GPU memory belongs to another allocator that reserved it up front, or they
must not risk an allocation failure or the synchronisation an allocation can
cause mid-work); thr_query_static keeps all of its scratch in one fixed
device array of the library.  Two calls in a row must each return exactly
what thr_query returns (the arithmetic is exact, so the tolerance is zero),
and sizes beyond the array's limits must be rejected.  This file runs last
(pytest collects it last) and also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import paper_1402_4466_gb300 as thr
import synth

pytestmark = pytest.mark.gpu


def test_static_scratch_query_matches_thr_query():
    import torch
    assert torch.cuda.is_available()
    r = (1 << 20) + 77
    words, _ = synth.many_criteria(21, 24, r)
    gw, goff = thr.encode_many(words, r)
    idx = thr.idx_build_rle(gw, goff, r)
    rng = np.random.default_rng(21)
    queries = [(list(range(24)), 2),
               (rng.integers(0, 24, size=40).tolist(), 7)]
    outs = [torch.zeros(idx.nwords + 1, dtype=torch.int64, device="cuda") for _ in queries]
    lens = [thr.thr_query_static(idx, ids, T, out) for (ids, T), out in zip(queries, outs)]
    for (ids, T), out, n in zip(queries, outs, lens):
        want = thr.thr_query(idx, ids, T)
        got = out[:n].cpu().numpy().view(np.uint64)
        assert n == len(want)
        assert np.array_equal(got, want)
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
