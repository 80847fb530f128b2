#!/usr/bin/env python
"""Benchmark of the GPU threshold (T-overlap) query.

Workload (the many-criteria configuration): 64 bitmaps over r = 2^26 rows,
densities log-uniform in [1e-4, 0.3], bitmaps 0-31 i.i.d. Bernoulli and
32-63 clustered (runs of mean 256 rows), encoded in the library's 64-bit
word-aligned run-length format (~125 MiB of compressed input).  One step runs
the four queries over all 64 bitmaps at T = 2, 16, 32 and 63.

Reported (one JSON line from rank 0):
  value         queries/s over the timed steps, index resident in HBM, output
                into a device pool; one step = the four queries as one
                thr_query_batch call (CUDA graph, autotuned launch, learned
                variant policy), timed with CUDA events around the call; L2 is
                flushed (256 MiB write, untimed) before every step
  plain         the same queries as one thr_query call each
  input_gbs     compressed input bytes / time (Sec. 7 of the paper measures
                throughput as input bytes over time)
  e2e           the same batch through the C ABI with host ids and a host
                result pool (the results copied back inside the timed call)
  roofline      the query kernel: algorithmic bytes (compressed input read +
                compressed output written) per launch / its event-timed
                duration, against the measured HBM copy bandwidth
  cpu_baseline  the CPU oracle on the same queries (bounded sample)

Multi-GPU (torchrun): every rank holds a full replica and runs the same
steps; value = all ranks' queries / the slowest rank's time ("weak").

--impl reference times the CPU oracle itself as the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = ("threshold queries/s and compressed-input GB/s (bit-exact) vs HBM peak; "
          "batched+learned vs plain")
WORKLOAD = ("many-criteria: 64 bitmaps x 2^26 rows, densities log-uniform [1e-4, 0.3], "
            "half i.i.d., half clustered (mean run 256 rows); one step = T in {2,16,32,63}")
KERNEL_SOURCES = ("thr_device.cuh", "thr_query_kernel.cuh", "thr_staged.cuh")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-query", type=int, default=None, metavar="T",
                    help="build the workload, run one warm-up query at threshold T and "
                         "then one more (the launch to capture with a profiler); no timing")
    ap.add_argument("--variant", default="csa",
                    choices=["csa", "staged", "position", "scancount", "looped"],
                    help="counting variant of --profile-query")
    ap.add_argument("--batch", action="store_true",
                    help="with --profile-query: the step's four thresholds as one batched "
                         "call (shared counting pass) instead of one query")
    ap.add_argument("--profile-opt", type=int, default=None, metavar="K",
                    help="like --profile-query for the opt-threshold query with K rows "
                         "(profiling pass, then the threshold query)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1402_4466_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic(which: str):
    """DRAM bytes per launch of a committed ncu capture ("t2", "t16", "t32",
    "t63": one query at that threshold; "step": the batched step's shared
    counting launch), if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "threshold_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(which)
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid: str | None):
        self.lines = []
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if device_uuid:
            cmd += ["-i", device_uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout=5.0):
        """Wait until nvidia-smi has printed its first sample."""
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_index_inputs(seed):
    import paper_1402_4466_gb300 as thr
    r = synth.MANY_R
    words, dens = synth.many_criteria(seed, synth.MANY_N, r,
                                      workers=min(16, os.cpu_count() or 1))
    gw, goff = thr.encode_many(words, r)
    return r, gw, goff


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1402_4466_gb300 as thr
    from paper_1402_4466_gb300 import selector_weights

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    stream = torch.cuda.Stream()
    r, gw, goff = make_index_inputs(args.seed)
    t0 = time.perf_counter()
    idx = thr.idx_build_rle(gw, goff, r, stream=stream)
    build_s = time.perf_counter() - t0
    ids = np.arange(synth.MANY_N, dtype=np.uint32)
    Ts = list(synth.MANY_TS)
    qs = [(ids, T) for T in Ts]
    in_bytes = 8 * int(goff[-1])  # every query reads all 64 streams
    W = idx.nwords
    dout = torch.empty(W + 1, dtype=torch.int64, device="cuda")
    pool = torch.empty(len(Ts) * (W + 1), dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    POLICY = thr.THR_POLICY_LEARNED
    sel = selector_weights.attach(idx)  # the shipped cost model (and refit rule)

    def flushed():
        with torch.cuda.stream(stream):
            flush.zero_()  # write 256 MiB > L2 before every timed call (untimed)
        stream.synchronize()

    out_words = {}
    last_step = {}

    def batched_step():
        """The step's four queries as one thr_query_batch call (CUDA graph,
        autotuned launch, learned variant policy); CUDA events on the
        caller's stream around the synchronous call."""
        flushed()
        ev0.record(stream)
        off, ln, _ = thr.thr_query_batch(idx, qs, pool=pool, flags=POLICY, stream=stream)
        ev1.record(stream)
        ev1.synchronize()
        for T, n in zip(Ts, ln):
            out_words[T] = int(n)
        last_step["off"], last_step["len"] = off.copy(), ln.copy()
        return ev0.elapsed_time(ev1)

    def batched_call(flags):
        flushed()
        ev0.record(stream)
        thr.thr_query_batch(idx, qs, pool=pool, flags=flags, stream=stream)
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1)

    def plain_query(T, flags=0, profile=True):
        """One thr_query (device output); CUDA events around the call, and
        with profile the pass-A kernel time (THR_PROFILE times each launch
        and so runs without the graph replay)."""
        flushed()
        ev0.record(stream)
        n = thr.thr_query(idx, ids, T, out=dout,
                          flags=flags | (thr.THR_PROFILE if profile else 0), stream=stream)
        ev1.record(stream)
        ev1.synchronize()
        out_words[T] = int(n)
        return ev0.elapsed_time(ev1), (thr.thr_last_kernel_ms() if profile else None)

    # launch configurations of this workload's shapes (autotuner)
    single_cfg, single_tune_ms = thr.thr_autotune(idx, [qs[0]], reps=3, stream=stream)
    batch_cfg, batch_tune_ms = thr.thr_autotune(idx, qs, flags=POLICY, reps=3, stream=stream)
    thr.thr_autotune(idx, qs, flags=POLICY | thr.THR_NO_SHARE, reps=3, stream=stream)

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)  # from the warm-up on, so that it has samples under load
    for _ in range(args.warmup):
        batched_step()
        for T in Ts:
            plain_query(T)
            plain_query(T, profile=False)
    clocks.wait_first()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    b_ms = [batched_step() for _ in range(args.steps)]
    binfo = thr.thr_last_batch_info()
    # the results of the last timed call, read back (untimed) for the oracle check
    pool_host = pool.cpu().numpy().view(np.uint64)
    timed_results = {T: pool_host[int(o): int(o) + int(n)].copy()
                     for T, o, n in zip(Ts, last_step["off"], last_step["len"])}
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = sum(b_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    nq = len(Ts) * args.steps * world
    value = nq / (total_ms / 1e3)
    input_gbs = (in_bytes * nq) / (total_ms / 1e3) / 1e9

    # the same batch without the shared counting pass (each query counts its
    # own inputs), and the pass-A time of the batched step (THR_PROFILE)
    nos_ms = [batched_call(POLICY | thr.THR_NO_SHARE) for _ in range(args.steps)]
    thr.thr_query_batch(idx, qs, pool=pool, flags=POLICY | thr.THR_PROFILE, stream=stream)
    step_pass_a_ms = thr.thr_last_kernel_ms()

    # plain: one thr_query per query (default variant, graph replay), and
    # in separate calls the pass-A kernel time of each (the roofline's launch)
    q_ms, k_ms_t = [], {T: [] for T in Ts}
    for _ in range(args.steps):
        for T in Ts:
            q_ms.append(plain_query(T, profile=False)[0])
            k_ms_t[T].append(plain_query(T)[1])
    plain_value = len(q_ms) / (sum(q_ms) / 1e3)
    plain_results = {T: thr.thr_query(idx, ids, T) for T in Ts}
    variant_ms = {}
    for vname, vflag in (("csa", thr.THR_VARIANT_CSA), ("staged", thr.THR_VARIANT_STAGED),
                         ("position", thr.THR_VARIANT_POSITION),
                         ("scancount", thr.THR_VARIANT_SCANCOUNT)):
        per_t = {}
        for T in Ts:
            ts = [plain_query(T, vflag)[1] for _ in range(max(args.steps, 3))]
            per_t[str(T)] = round(statistics.median(ts), 5)
        variant_ms[vname] = per_t
    # Looped levels (T <= 4 only; T = 1 and 2 on these bitmaps) next to carry-save
    saved_out = dict(out_words)
    variant_ms["looped_vs_csa"] = {
        str(T): {v: round(statistics.median(
            [plain_query(T, f)[1] for _ in range(max(args.steps, 3))]), 5)
            for v, f in (("looped", thr.THR_VARIANT_LOOPED), ("csa", thr.THR_VARIANT_CSA))}
        for T in (1, 2)}
    out_words.clear()
    out_words.update(saved_out)
    # symmetric functions of the same counts (at most 1, exactly 2, 2..4, odd)
    sym_ms = {}
    for name, lo, hi, odd in (("at_most_1", 0, 1, False), ("exactly_2", 2, 2, False),
                              ("between_2_4", 2, 4, False), ("odd", 0, 0, True)):
        ts = []
        for _ in range(max(args.steps, 3)):
            flushed()
            thr.thr_query_sym(idx, ids, lo, hi, odd=odd, out=dout, stream=stream,
                              flags=thr.THR_PROFILE)
            ts.append(thr.thr_last_kernel_ms())
        sym_ms[name] = round(statistics.median(ts), 5)
    # opt-threshold (largest T with K rows): the profiling pass alone, and the
    # whole call (profiling pass, histogram read, threshold query at T)
    opt = {}
    for K in (1, 1000):
        prof, whole, Tk = [], [], 0
        for _ in range(max(args.steps, 3)):
            flushed()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            Tk, _ = thr.thr_query_opt(idx, ids, K, out=dout, stream=stream,
                                      flags=thr.THR_PROFILE)
            whole.append((time.perf_counter() - t1) * 1e3)
            prof.append(thr.thr_last_kernel_ms())
        opt[f"K={K}"] = {"T": int(Tk), "profile_ms": round(statistics.median(prof), 5),
                         "call_ms": round(statistics.median(whole), 5)}
    clk = clocks.stop()

    # end to end through the C ABI: host ids in, host result pool out (the
    # pool is page-locked host memory allocated once and reused, as a caller
    # streaming results would; its pages are touched before timing)
    host_pool = torch.zeros(len(Ts) * (W + 1), dtype=torch.int64, pin_memory=True)
    thr.thr_query_batch(idx, qs, pool=host_pool, flags=POLICY, stream=stream)
    e2e_ms, d2h = [], 0
    for _ in range(args.steps):
        flushed()
        t1 = time.perf_counter()
        off, ln, hp = thr.thr_query_batch(idx, qs, pool=host_pool, flags=POLICY, stream=stream)
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
        d2h += 8 * int(ln.sum()) + 16 * len(Ts)
    e2e_value = len(Ts) * len(e2e_ms) / (sum(e2e_ms) / 1e3)
    hp_host = hp.numpy().view(np.uint64)
    e2e_results = {T: hp_host[int(o): int(o) + int(n)].copy() for T, o, n in zip(Ts, off, ln)}
    plain_cfg = plain_workload(thr, torch, stream, args)

    peak, peak_kind = measured_peaks()
    by_t = {}
    for T in Ts:
        b = in_bytes + 8 * out_words[T]
        km = statistics.median(k_ms_t[T])
        by_t[str(T)] = {"bytes": b, "kernel_ms": round(km, 5),
                        "achieved_gbs": round(b / (km / 1e3) / 1e9, 1),
                        "frac": round(b / (km / 1e3) / 1e9 / peak, 4),
                        "traffic": ncu_traffic(f"t{T}")}
    # the headline: the dense, low-threshold launch (T = 2), where the bytes
    # credited are the bytes the kernel has to read
    dense = by_t[str(Ts[0])]
    step_moved = ncu_traffic("step")
    launches_per_step = binfo["launches"] + 2 * binfo["chunks"]
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "queries/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u64",
        "data": "synthetic",
        "input_gbs": round(input_gbs, 2),
        "config": {
            "workload": WORKLOAD,
            "bitmaps": synth.MANY_N,
            "rows": r,
            "thresholds": Ts,
            "compressed_input_bytes_per_query": in_bytes,
            "output_words": {str(k): int(v) for k, v in out_words.items()},
            "step": "the four queries as one thr_query_batch call: CUDA graph replay, "
                    "autotuned launch, learned variant policy (shipped cost model)",
            "l2": "flushed before every timed call (256 MiB device write, untimed)",
            "parallelism": f"replicas x{world}",
            "index_build_s": round(build_s, 3),
        },
        "e2e": {"value": round(e2e_value, 3), "unit": "queries/s",
                "h2d_bytes_per_step": 4 * len(ids) * len(Ts) + 8 * (len(Ts) + 1),
                "d2h_bytes_per_step": d2h // max(args.steps, 1)},
        "plain": {"value": round(plain_value, 3), "unit": "queries/s",
                  "what": "one thr_query per query (device output, default variant, CUDA "
                          "graph replayed), CUDA events around each call",
                  "batched_speedup": round(value / plain_value, 3)},
        "batched_without_sharing": {
            "value": round(len(Ts) * len(nos_ms) / (sum(nos_ms) / 1e3), 3), "unit": "queries/s",
            "what": "the same batched call with THR_NO_SHARE: every query counts its own "
                    "inputs (the default shares one counting pass among queries over the "
                    "same id multiset)"},
        "roofline_step": {
            "what": "pass A of the batched step: one launch counting the four queries' "
                    "shared inputs once; credited = every query's input and output bytes, "
                    "moved = DRAM bytes of one launch (ncu, null when taken on other "
                    "kernel sources)",
            "pass_a_ms": round(step_pass_a_ms, 5),
            "credited_bytes": 4 * in_bytes + 8 * sum(out_words.values()),
            "credited_frac": round((4 * in_bytes + 8 * sum(out_words.values())) /
                                   (step_pass_a_ms / 1e3) / 1e9 / peak, 4),
            "moved_bytes": step_moved,
            "moved_frac": (round(step_moved / (step_pass_a_ms / 1e3) / 1e9 / peak, 4)
                           if step_moved else None),
            "input_bytes_read_once": in_bytes},
        "roofline": {"bound": "hbm", "achieved": dense["achieved_gbs"], "peak": peak,
                     "unit": "GB/s", "frac": dense["frac"],
                     "traffic": ncu_traffic("t2"), "peak_kind": peak_kind,
                     "kernel": "pass A (k_threshold family), one query at T = %d" % Ts[0],
                     "bytes_per_launch": dense["bytes"], "kernel_ms": dense["kernel_ms"],
                     "launch_config": single_cfg, "by_threshold": by_t},
        "batched": {"launch_config": binfo["config"], "graph_replayed": binfo["graph"] == 1,
                    "pass_a_launches": binfo["launches"], "chunks": binfo["chunks"],
                    "variants": thr.select_variants(idx, qs, POLICY).tolist(),
                    "autotune_ms": [round(t, 4) for t in batch_tune_ms],
                    "single_query_autotune_ms": [round(t, 4) for t in single_tune_ms]},
        "pass_a_ms_by_variant": variant_ms,
        "pass_a_ms_symmetric": sym_ms,
        "opt_threshold": opt,
        "plain_workload": plain_cfg,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(
            gw, goff, r, ids, Ts, {"timed_batched_path": timed_results,
                                   "e2e_host_pool": e2e_results,
                                   "plain_thr_query": plain_results})
    if rank == 0:
        print(json.dumps(line), flush=True)
    thr.set_selector(idx, None)
    del sel
    idx.close()
    if world > 1:
        dist.destroy_process_group()


def time_until(fn, min_total_s=1.0, max_reps=50):
    """Run fn repeatedly until the runs add up to min_total_s (the paper's
    protocol, Sec. 7: repeat until at least one second); seconds per run."""
    ts = []
    while sum(ts) < min_total_s and len(ts) < max_reps:
        t0 = time.perf_counter()
        fn()
        ts.append(time.perf_counter() - t0)
    return ts


def cpu_baseline(gw, goff, r, ids, Ts, gpu_results):
    """The oracle (plain ScanCount) on the step's 4 queries: single-threaded,
    and row-partitioned over every host core (OpenMP); each query repeated
    until its runs add up to 1 s, min and median reported.  The GPU results
    of the timed batched call, of the end-to-end call and of plain
    thr_query calls are compared word for word with the oracle's."""
    import oracle
    streams = [gw[int(goff[i]): int(goff[i + 1])] for i in range(len(goff) - 1)]
    o = oracle.Index(streams, r)
    cores = oracle.load().max_threads()
    single, multi, want = [], [], {}
    for T in Ts:
        want[T] = o.threshold(ids, T)
        single += time_until(lambda: o.threshold(ids, T))
        multi += time_until(lambda: o.threshold_parts(ids, T, cores))
        assert np.array_equal(o.threshold_parts(ids, T, cores), want[T])
    match = {k: all(np.array_equal(v[T], want[T]) for T in Ts) for k, v in gpu_results.items()}
    med = statistics.median(multi)
    return {"value": round(1.0 / med, 4), "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": "the 4 queries of one step (T = 2, 16, 32, 63), each repeated until 1 s; "
                      "rows partitioned over every host core (OpenMP); value = 1 / median",
            "min_s": round(min(multi), 4), "median_s": round(med, 4),
            "single_thread": {"value": round(1.0 / statistics.median(single), 4),
                              "unit": "queries/s", "cores": 1,
                              "min_s": round(min(single), 4),
                              "median_s": round(statistics.median(single), 4)},
            "gpu_matches_oracle": all(match.values()), "checked": match}


def plain_workload(thr, torch, stream, args):
    """The plain single query (8 Bernoulli(0.05) bitmaps over 2^20 rows,
    T = 4; about 1 MiB of input, which stays in L2): latency of one
    thr_query call (device output, synchronous) and the rate of calls one
    after another, checked against the oracle."""
    import oracle
    words = synth.plain(0, synth.PLAIN_N, synth.PLAIN_R, synth.PLAIN_P)
    gw, goff = thr.encode_many(words, synth.PLAIN_R)
    idx = thr.idx_build_rle(gw, goff, synth.PLAIN_R, stream=stream)
    ids = np.arange(synth.PLAIN_N, dtype=np.uint32)
    dout = torch.empty(idx.nwords + 1, dtype=torch.int64, device="cuda")
    for _ in range(20):
        thr.thr_query(idx, ids, synth.PLAIN_T, out=dout, stream=stream)
    lat = []
    for _ in range(max(200, 20 * args.steps)):
        t0 = time.perf_counter()
        n = thr.thr_query(idx, ids, synth.PLAIN_T, out=dout, stream=stream)
        lat.append((time.perf_counter() - t0) * 1e3)
    got = dout[:n].cpu().numpy().view(np.uint64)
    o = oracle.Index([oracle.encode(w, synth.PLAIN_R) for w in words], synth.PLAIN_R)
    ok = bool(np.array_equal(got, o.threshold(ids, synth.PLAIN_T)))
    thr.thr_query(idx, ids, synth.PLAIN_T, out=dout, stream=stream, flags=thr.THR_PROFILE)
    km = thr.thr_last_kernel_ms()
    idx.close()
    lat.sort()
    return {"workload": "plain: 8 Bernoulli(0.05) bitmaps x 2^20 rows, T = 4 (input in L2)",
            "compressed_input_bytes": 8 * int(goff[-1]),
            "queries_per_s": round(len(lat) / (sum(lat) / 1e3), 1),
            "latency_ms_p50": round(lat[len(lat) // 2], 4),
            "latency_ms_p99": round(lat[int(0.99 * (len(lat) - 1))], 4),
            "pass_a_ms": round(km, 5), "matches_oracle": ok}


def run_reference(args):
    """The CPU oracle as the reference arm: every query of a step runs the
    row-partitioned ScanCount over all host cores (OpenMP), one query after
    another."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    r = synth.MANY_R
    words, _ = synth.many_criteria(args.seed, synth.MANY_N, r,
                                   workers=min(16, os.cpu_count() or 1))
    streams = [oracle.encode(w, r) for w in words]
    o = oracle.Index(streams, r)
    cores = oracle.load().max_threads()
    ids = np.arange(synth.MANY_N, dtype=np.uint32)
    Ts = list(synth.MANY_TS)

    def step():
        for T in Ts:
            o.threshold_parts(ids, T, cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = len(Ts) * args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "queries/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "bitmaps": synth.MANY_N, "rows": r, "thresholds": Ts},
        "cpu_baseline": {"value": round(value, 4), "unit": "queries/s", "cores": cores,
                         "kind": "oracle",
                         "sample": "every step: the 4 queries one after another, each "
                                   "row-partitioned over every host core (OpenMP)"},
        "e2e": {"value": round(value, 4), "unit": "queries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def profile_query(args):
    """One warm-up query and one captured query of the many-criteria workload
    (for ncu: the second launch of each kernel is the one to capture)."""
    import torch

    import paper_1402_4466_gb300 as thr
    torch.cuda.init()
    r, gw, goff = make_index_inputs(args.seed)
    idx = thr.idx_build_rle(gw, goff, r)
    flag = {"csa": thr.THR_VARIANT_CSA, "staged": thr.THR_VARIANT_STAGED,
            "position": thr.THR_VARIANT_POSITION,
            "scancount": thr.THR_VARIANT_SCANCOUNT, "looped": thr.THR_VARIANT_LOOPED}[args.variant]
    ids = np.arange(synth.MANY_N, dtype=np.uint32)
    dout = torch.empty(idx.nwords + 1, dtype=torch.int64, device="cuda")
    pool = torch.empty(4 * (idx.nwords + 1), dtype=torch.int64, device="cuda")
    for _ in range(2):
        if args.profile_opt is not None:
            T, n = thr.thr_query_opt(idx, ids, args.profile_opt, out=dout)
        elif args.batch:
            _, ln, _ = thr.thr_query_batch(idx, [(ids, T) for T in synth.MANY_TS], pool=pool,
                                           flags=flag | thr.THR_NO_GRAPH)
            n = int(ln.sum())
        else:
            n = thr.thr_query(idx, ids, args.profile_query, out=dout, flags=flag)
    torch.cuda.synchronize()
    print(json.dumps({"profile_query": args.profile_query, "variant": args.variant,
                      "output_words": n, "input_bytes": 8 * int(goff[-1])}))
    idx.close()


def main():
    args = parse()
    if args.profile_query is not None or args.profile_opt is not None:
        profile_query(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
