"""Batched similarity queries: 4096 threshold queries of uneven size in one
thr_query_batch call against the plain per-query launch.

Workload (``workloads.similarity``): 2^16 term bitmaps over 2^24 documents,
term densities min(0.3, C k^-1.1) summing to 110; each query takes the
N ~ U[10, 200] Zipf-drawn terms of a document, whose prototype row is
planted in those bitmaps, with T = ceil(N / 2).

Timed (host wall clock around each synchronous call, L2 flushed before it;
inputs resident in HBM, results into a device pool):
  plain     one thr_query per query (default variant, launch configuration
            of a single query)
  batched   the 4096 queries in one thr_query_batch call (CUDA graph, launch
            configuration from the autotuner), with the plain, rule and
            learned variant policies
Checked: every sampled batched result equals the plain one (word for
word) and contains its query's prototype row.  (The comparison with the CPU
oracle at this workload's shape is a GPU test, tests/test_gpu_configs.py.)

    python -m paper_1402_4466_gb300.batch_bench --out similarity.json
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_1402_4466_gb300 as thr  # noqa: E402
from paper_1402_4466_gb300 import workloads  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nb", type=int, default=1 << 16)
    ap.add_argument("--log-r", type=int, default=24)
    ap.add_argument("--queries", type=int, default=4096)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--pool", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    import torch
    torch.cuda.init()
    t0 = time.time()
    words, offsets, r, queries, protos = workloads.similarity(args.nb, 1 << args.log_r,
                                                              args.queries, 0, args.pool)
    gen_s = time.time() - t0
    t0 = time.time()
    idx = thr.idx_build_rle(words, offsets, r)
    build_s = time.time() - t0
    lens = np.diff(offsets.astype(np.int64))
    in_bytes = [8 * int(lens[ids].sum()) for ids, _ in queries]
    W = idx.nwords
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    dout = torch.empty(W + 1, dtype=torch.int64, device="cuda")

    def flushed(fn):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        t1 = time.perf_counter()
        out = fn()
        return (time.perf_counter() - t1) * 1e3, out

    # plain: one query at a time
    def plain():
        lens_out = []
        for ids, T in queries:
            lens_out.append(thr.thr_query(idx, ids, T, out=dout, stream=stream))
        return lens_out

    plain()  # warm-up
    p_ms = [flushed(plain)[0] for _ in range(args.reps)]

    # batched: autotune the launch configuration on a sample, then the batch
    tune_best, tune_ms = thr.thr_autotune(idx, queries[:512], reps=2, stream=stream)
    pool = torch.empty(len(queries) * (W + 1), dtype=torch.int64, device="cuda")
    sel = None
    try:
        from paper_1402_4466_gb300 import selector_weights
        sel = selector_weights.attach(idx)
    except FileNotFoundError:
        sel = None
    results = {}
    for name, flags in (("plain", thr.THR_POLICY_PLAIN), ("rule", thr.THR_POLICY_RULE),
                        ("learned", thr.THR_POLICY_LEARNED)):
        def batch():
            return thr.thr_query_batch(idx, queries, pool=pool, flags=flags, stream=stream)
        batch()  # warm-up (graph instantiation)
        ms = []
        for _ in range(args.reps):
            t, (off, ln, _) = flushed(batch)
            ms.append(t)
        info = thr.thr_last_batch_info()
        variants = thr.select_variants(idx, queries, flags)
        results[name] = {"ms": [round(x, 3) for x in ms],
                         "qps": round(len(queries) / (min(ms) / 1e3), 1),
                         "input_gbs": round(sum(in_bytes) / (min(ms) / 1e3) / 1e9, 1),
                         "chunks": info["chunks"], "pass_a_launches": info["launches"],
                         "launch_config": info["config"], "graph_replayed": info["graph"] == 1,
                         "variant_counts": np.bincount(variants, minlength=3).tolist()}
        print(json.dumps({name: results[name]}), flush=True)

    # checks: batch == plain, prototype rows present
    off, ln, _ = thr.thr_query_batch(idx, queries, pool=pool, stream=stream)
    host = pool.cpu().numpy().view(np.uint64)
    mismatches = 0
    proto_missing = 0
    sampled = range(0, len(queries), 16)
    for k in sampled:
        ids, T = queries[k]
        got = host[int(off[k]): int(off[k] + ln[k])]
        mismatches += 0 if np.array_equal(got, thr.thr_query(idx, ids, T)) else 1
        # the prototype row lies in every input, hence in the result (T <= N)
        w_i, b_i = divmod(protos[k], 64)
        pos = 0
        i = 0
        while i < len(got):  # expand only up to the prototype's word
            m = int(got[i])
            F, L, fb = (m >> 1) & 0xFFFFFFFF, m >> 33, m & 1
            if pos + F > w_i:
                bit = fb
                break
            pos += F
            if pos + L > w_i:
                bit = (int(got[i + 1 + (w_i - pos)]) >> b_i) & 1
                break
            pos += L
            i += 1 + L
        else:
            bit = 0
        proto_missing += 0 if bit else 1
    res = {
        "workload": f"similarity: {args.nb} term bitmaps x 2^{args.log_r} rows, densities "
                    f"min(0.3, C k^-1.1) summing to 110, {len(queries)} queries of N~U[10,200] "
                    f"Zipf-drawn terms with a planted prototype row, T=ceil(N/2)",
        "index_words": int(offsets[-1]), "generate_s": round(gen_s, 1),
        "index_build_s": round(build_s, 1),
        "mean_input_mib_per_query": round(np.mean(in_bytes) / 2 ** 20, 1),
        "plain": {"ms": [round(x, 3) for x in p_ms],
                  "qps": round(len(queries) / (min(p_ms) / 1e3), 1),
                  "input_gbs": round(sum(in_bytes) / (min(p_ms) / 1e3) / 1e9, 1)},
        "batched": results,
        "autotune": {"best": tune_best, "ms": [round(x, 3) for x in tune_ms]},
        "checks": {"sampled": len(sampled), "batch_vs_plain_mismatches": mismatches,
                   "prototype_rows_missing": proto_missing},
    }
    res["speedup_batched_learned_vs_plain"] = round(results["learned"]["qps"] /
                                                    res["plain"]["qps"], 3)
    print(json.dumps(res), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)
    idx.close()


if __name__ == "__main__":
    main()
