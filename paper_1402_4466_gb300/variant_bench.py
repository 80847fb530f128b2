"""Pass-A time of the counting variants on very sparse inputs, the regime
ScanCount is made for (Sec. 5.1: one counter increment per set bit, so its
cost follows the set bits, while carry-save counting costs the literal words
times the counter slices, and the slices grow with log2 T).

Workload (``workloads.sparse``): nb i.i.d. Bernoulli(p) bitmaps over r rows
(defaults 4096, 2^24, 2e-4: about 3,400 set rows per bitmap, one or two
literal words per bitmap in most 8,192-row subtiles).  Queries take the
first n bitmaps, n in 256 / 1024 / 4096, at thresholds T in 2 / 8 / 32 / 128
(T <= n).  Per (n, T) and variant (grouped carry-save, ScanCount with 8- or
16-bit counters, position lists): the median pass-A kernel time over reps
single-query calls with L2 flushed before each, the variants the rule and
learned choosers pick, and the result of every variant checked against the
definition of Sec. 2 (rows counted at least T times, from the row lists).

    python -m paper_1402_4466_gb300.variant_bench --out sparse_variants.json
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_1402_4466_gb300 as thr  # noqa: E402
import synth  # noqa: E402
from paper_1402_4466_gb300 import workloads  # noqa: E402

VARIANTS = (("csa", thr.THR_VARIANT_CSA), ("scancount", thr.THR_VARIANT_SCANCOUNT),
            ("position", thr.THR_VARIANT_POSITION))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nb", type=int, default=4096)
    ap.add_argument("--log-r", type=int, default=24)
    ap.add_argument("--density", type=float, default=2e-4)
    ap.add_argument("--ns", default="256,1024,4096")
    ap.add_argument("--ts", default="2,8,32,128")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--pool", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    import torch
    torch.cuda.init()
    r = 1 << args.log_r
    t0 = time.time()
    words, offsets = workloads.sparse(args.nb, r, args.density, 0, args.pool)
    gen_s = time.time() - t0
    idx = thr.idx_build_rle(words, offsets, r)
    from paper_1402_4466_gb300 import selector_weights
    sel = selector_weights.attach(idx)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    dout = torch.empty(idx.nwords + 1, dtype=torch.int64, device="cuda")
    lens = np.diff(offsets.astype(np.int64))
    ns = [int(x) for x in args.ns.split(",") if int(x) <= args.nb]
    ts = [int(x) for x in args.ts.split(",")]
    # per-row counts of every prefix of the bitmaps (the definition's side)
    counts = np.zeros(r, np.int32)
    done = 0
    res = {"workload": f"sparse: {args.nb} Bernoulli({args.density}) bitmaps over 2^{args.log_r} "
                       "rows; queries over the first n bitmaps",
           "index_words": int(offsets[-1]), "generate_s": round(gen_s, 1),
           "timing": f"pass-A kernel time (THR_PROFILE), median of {args.reps} single-query "
                     "calls, L2 flushed (256 MiB write) before each",
           "cases": []}
    try:
        for n in ns:
            for k in range(done, n):
                counts[synth.bitmap_rows(0, k, r, args.density, False)] += 1
            done = n
            ids = np.arange(n, dtype=np.uint32)
            for T in ts:
                if T > n:
                    continue
                want = thr.thr_rle_encode_rows(np.nonzero(counts >= T)[0], r)
                case = {"n": n, "T": T, "input_bytes": 8 * int(lens[:n].sum()),
                        "rows": int((counts >= T).sum()), "pass_a_ms": {}, "matches": {}}
                for name, flag in VARIANTS:
                    got = thr.thr_query(idx, ids, T, flags=flag)
                    case["matches"][name] = bool(np.array_equal(got, want))
                    tms = []
                    for _ in range(args.reps):
                        with torch.cuda.stream(stream):
                            flush.zero_()
                        stream.synchronize()
                        thr.thr_query(idx, ids, T, out=dout, flags=flag | thr.THR_PROFILE,
                                      stream=stream)
                        tms.append(thr.thr_last_kernel_ms())
                    case["pass_a_ms"][name] = round(statistics.median(tms), 5)
                best = min(case["pass_a_ms"], key=case["pass_a_ms"].get)
                case["fastest"] = best
                case["scancount_speedup_vs_csa"] = round(
                    case["pass_a_ms"]["csa"] / case["pass_a_ms"]["scancount"], 3)
                names = {0: "csa", 1: "position", 2: "scancount", 3: "split"}
                for pol, f in (("rule", thr.THR_POLICY_RULE), ("learned", thr.THR_POLICY_LEARNED)):
                    case[f"{pol}_picks"] = names.get(
                        int(thr.select_variants(idx, [(ids, T)], f)[0]), "?")
                res["cases"].append(case)
                print(json.dumps(case), flush=True)
    finally:
        thr.set_selector(idx, None)
        del sel
        idx.close()
    print(json.dumps(res), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
