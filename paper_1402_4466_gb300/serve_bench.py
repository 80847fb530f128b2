"""Serving benchmark: Poisson arrivals of threshold queries against a
resident index, served with continuous batching (thr_server_*).

Workload (defaults): the serving index of ``workloads.serving`` (2^14
bitmaps over 2^26 rows, Zipf(1.1) densities, odd i.i.d., even clustered);
each query draws N uniform in 3..256 bitmap ids (uniform, with replacement)
and T uniform in 1..N.  For every arrival rate a submitter thread releases
the queries at exponential inter-arrival times; the latency of a query is
from its scheduled arrival to the completion of its result (queueing in the
submitter included).  Reported per rate: offered and sustained queries/s,
p50 / p99 / max latency, and the server's batch statistics; then a closed
burst (every query submitted at once) gives the saturated throughput.

    python -m paper_1402_4466_gb300.serve_bench --rates 2000,8000,32000
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_1402_4466_gb300 as thr  # noqa: E402
from paper_1402_4466_gb300 import workloads  # noqa: E402


def draw_queries(seed, count, nb):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(3, 257))
        out.append((rng.integers(0, nb, n).astype(np.uint32), int(rng.integers(1, n + 1))))
    return out


def run_rate(srv, queries, rate, seed):
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(queries)))
    tickets = [None] * len(queries)
    lag = np.zeros(len(queries))
    t0 = time.perf_counter()

    def submitter():
        for i, (ids, T) in enumerate(queries):
            wait = arrivals[i] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            lag[i] = max(0.0, (time.perf_counter() - t0) - arrivals[i])
            tickets[i] = srv.submit(ids, T)

    th = threading.Thread(target=submitter)
    th.start()
    lat = np.zeros(len(queries))
    for i in range(len(queries)):
        while tickets[i] is None:
            time.sleep(0.0002)
        _, ms = srv.wait(tickets[i])
        lat[i] = ms + 1e3 * lag[i]
    th.join()
    elapsed = time.perf_counter() - t0
    return lat, elapsed, arrivals[-1]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nb", type=int, default=1 << 14)
    ap.add_argument("--log-r", type=int, default=26)
    ap.add_argument("--rates", default="1000,4000,16000,64000")
    ap.add_argument("--queries", type=int, default=4000, help="queries per rate")
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--max-batch", type=int, default=64)
    ap.add_argument("--budget-gb", type=float, default=8.0)
    ap.add_argument("--policy", default="rule", choices=["plain", "rule", "learned"])
    ap.add_argument("--pool", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    import torch
    torch.cuda.init()
    t0 = time.time()
    words, offsets, r = workloads.serving(args.nb, 1 << args.log_r, 0, args.pool)
    idx = thr.idx_build_rle(words, offsets, r)
    build_s = time.time() - t0
    flags = {"plain": thr.THR_POLICY_PLAIN, "rule": thr.THR_POLICY_RULE,
             "learned": thr.THR_POLICY_LEARNED}[args.policy]
    if args.policy == "learned":
        from paper_1402_4466_gb300 import selector_weights
        selector_weights.attach(idx)
    srv = thr.Server(idx, workers=args.workers, max_batch=args.max_batch,
                     mem_budget=int(args.budget_gb * (1 << 30)), flags=flags)
    # warm-up: graphs, pools, selector
    warm = draw_queries(99, 200, args.nb)
    for t in [srv.submit(ids, T) for ids, T in warm]:
        srv.wait(t)
    res = {"workload": f"serving: {args.nb} bitmaps x 2^{args.log_r} rows, Zipf(1.1) densities "
                       f"0.3 k^-1.1 (odd i.i.d., even clustered); N ~ U[3,256], T ~ U[1,N]",
           "index_words": int(offsets[-1]), "index_build_s": round(build_s, 1),
           "workers": args.workers, "max_batch": args.max_batch, "budget_gb": args.budget_gb,
           "policy": args.policy, "rates": []}
    for i, rate in enumerate(float(x) for x in args.rates.split(",")):
        qs = draw_queries(1000 + i, args.queries, args.nb)
        before = srv.stats()
        lat, elapsed, span = run_rate(srv, qs, rate, 2000 + i)
        after = srv.stats()
        nb = after["batches"] - before["batches"]
        res["rates"].append({
            "offered_qps": rate,
            "sustained_qps": round(len(qs) / elapsed, 1),
            "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "max_ms": round(float(lat.max()), 3),
            "mean_batch": round((after["batched_queries"] - before["batched_queries"]) / max(nb, 1), 2),
            "max_in_flight": after["max_in_flight"],
        })
        print(json.dumps(res["rates"][-1]), flush=True)
    # saturated: everything at once
    qs = draw_queries(5000, args.queries, args.nb)
    t1 = time.perf_counter()
    tickets = [srv.submit(ids, T) for ids, T in qs]
    lat = np.array([srv.wait(t)[1] for t in tickets])
    el = time.perf_counter() - t1
    res["burst"] = {"queries": len(qs), "qps": round(len(qs) / el, 1),
                    "p50_ms": round(float(np.percentile(lat, 50)), 3),
                    "p99_ms": round(float(np.percentile(lat, 99)), 3)}
    res["server_stats"] = srv.stats()
    srv.close()
    idx.close()
    print(json.dumps(res), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
