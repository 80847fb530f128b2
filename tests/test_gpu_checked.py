"""The checked build (libthr_checked.so, selected with THR_CHECKED=1): the
same query paths with every index-derived access of the query kernels
compared with the size of what it addresses.  In a child process (the
library is loaded once per process): a mixed index (ragged tail, empty and
full bitmaps, clustered and i.i.d. inputs), batches under every counting
variant and both choosers, single, symmetric and static queries, and the
server with several workers under the learned policy -- each result equal to
the CPU oracle's (the plain definition of Sec. 2), and no check failing
(a failure would return THR_E_CHECK and raise)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
import oracle
import synth
import paper_1402_4466_gb300 as thr
from paper_1402_4466_gb300 import selector_weights

assert thr.checked() and thr.library_path().endswith("libthr_checked.so")
torch.cuda.init()
r = 3 * 8192 * 4 + 4100
rng = np.random.default_rng(12)
arrays = []
for i in range(48):
    if i == 0:
        arrays.append(np.zeros(synth.nwords(r), np.uint64))
    elif i == 1:
        arrays.append(synth.rows_to_words(np.arange(r), r))
    elif i % 3 == 0:
        arrays.append(synth.clustered(12, i, r, float(10 ** rng.uniform(-3, -0.3))))
    else:
        arrays.append(synth.bernoulli(12, i, r, float(10 ** rng.uniform(-4, -0.2))))
gw, goff = thr.encode_many(arrays, r)
g = thr.idx_build_rle(gw, goff, r)
o = oracle.Index([oracle.encode(a, r) for a in arrays], r)
sel = selector_weights.attach(g)
qs = []
for k in range(60):
    n = int(rng.integers(1, 300))
    ids = rng.integers(0, 48, n).astype(np.uint32)
    qs.append((ids, int(rng.integers(0, n + 2))))
qs.append((qs[3][0], qs[3][1] + 1))  # a group over one id multiset
want = [o.threshold(ids, T) for ids, T in qs]
flags = (0, thr.THR_VARIANT_SCANCOUNT, thr.THR_VARIANT_POSITION, thr.THR_VARIANT_SPLIT,
         thr.THR_VARIANT_LOOPED, thr.THR_VARIANT_STAGED, thr.THR_POLICY_RULE,
         thr.THR_POLICY_LEARNED, thr.THR_POLICY_LEARNED | thr.THR_NO_SHARE)
for fl in flags:
    off, ln, pool = thr.thr_query_batch(g, qs, flags=fl)
    for k in range(len(qs)):
        assert np.array_equal(pool[int(off[k]): int(off[k] + ln[k])], want[k]), (fl, k)
for k in range(0, len(qs), 7):
    ids, T = qs[k]
    assert np.array_equal(thr.thr_query(g, ids, T), want[k])
    lo, hi = max(T - 2, 0), T + 1
    c = np.stack([synth.words_to_bits(arrays[b], r) for b in ids]).sum(axis=0)
    rows = np.nonzero((c >= lo) & (c <= hi))[0]
    assert np.array_equal(thr.thr_query_sym(g, ids, lo, hi),
                          oracle.encode(synth.rows_to_words(rows, r), r))
    out = torch.empty(g.nwords + 1, dtype=torch.int64, device="cuda")
    n = thr.thr_query_static(g, ids, T, out)
    assert np.array_equal(out[:n].cpu().numpy().view(np.uint64), want[k])
srv = thr.Server(g, workers=4, max_batch=8, flags=thr.THR_POLICY_LEARNED)
try:
    tickets = [srv.submit(ids, T) for ids, T in qs * 3]
    for k, t in enumerate(tickets):
        res, _ = srv.wait(t)
        assert np.array_equal(res, want[k % len(qs)]), k
finally:
    srv.close()
thr.set_selector(g, None)
g.close()
print("checked build: all results equal the oracle, no check failed")
'''


def test_checked_build_matches_oracle_without_a_failed_check():
    env = dict(os.environ, THR_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True,
                       text=True, timeout=1800, cwd=ROOT)
    assert r.returncode == 0, (r.stdout[-4000:], r.stderr[-4000:])
    assert "no check failed" in r.stdout
