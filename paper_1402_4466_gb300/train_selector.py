"""Train the learned variant selector on timings the kernels produce.

Workloads: the plain and the many-criteria bitmap generators (module
``synth``) at r = 2^18 .. 2^26 rows, 256 bitmaps each, and very sparse
inputs: 1024 i.i.d. bitmaps per r with densities log-uniform in
[5e-5, 2e-3].  A query draws the family (plain 0.4, many-criteria 0.4,
sparse 0.2), r = 2^U{18..26}, N log-uniform in [3, 256] (sparse: [3, 1024]),
T uniform in 1..N and N ids with replacement; a query whose result is
empty is drawn again (at most 20 times).  Its label is, per counting
variant, the minimum pass-A time of `reps` runs after one warm-up
(THR_PROFILE), in ms; a variant that would fall back to the carry-save
kernel for the query (split above 8 counter bits) is masked out.

Then: features (thr_query_features), normalisation, training of the MLP with
the library's CUDA kernels (Adam on the squared error of log time), a least
squares refit of the rule chooser's time models (Sec. 8.1 form), and an
evaluation on held-out queries of four choosers against the measured best:
the learned model, the refit rule, the fixed carry-save default, and the
best single variant.

Writes (to --out): selector_weights.json (parameters, normalisation, rule
coefficients), selector_eval.json (the comparison) and selector_heldout.npz
(held-out features and measured times).

    python -m paper_1402_4466_gb300.train_selector --out selector_out
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

import paper_1402_4466_gb300 as thr  # noqa: E402
from paper_1402_4466_gb300 import workloads  # noqa: E402

NB = 256
NB_SPARSE = 1024
VARIANTS = ("csa", "position", "scancount", "split")


def _gen_plain(args):
    seed, k, r = args
    return synth.bernoulli(seed, k, r, synth.PLAIN_P)


def _gen_many(args):
    seed, k, r, p, clustered = args
    return synth.clustered(seed, k, r, p) if clustered else synth.bernoulli(seed, k, r, p)


def build_indexes(seed, log_rs, workers):
    """Two indexes per r: plain (Bernoulli 0.05) and many-criteria."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    out = {}
    ctx = mp.get_context("spawn")
    with ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
        for lr in log_rs:
            r = 1 << lr
            plain = list(ex.map(_gen_plain, [(seed + lr, k, r) for k in range(NB)]))
            dens = synth.log_uniform_densities(seed + 100 + lr, NB)
            many = list(ex.map(_gen_many, [(seed + 100 + lr, k, r, float(dens[k]), k >= NB // 2)
                                           for k in range(NB)]))
            for name, words in (("plain", plain), ("many", many)):
                gw, goff = thr.encode_many(words, r)
                out[(name, lr)] = thr.idx_build_rle(gw, goff, r)
            sd = synth.log_uniform_densities(seed + 200 + lr, NB_SPARSE, 5e-5, 2e-3)
            gw, goff = workloads.encode_family(
                [(seed + 200 + lr, k, r, float(sd[k]), False, None) for k in range(NB_SPARSE)],
                workers)
            out[("sparse", lr)] = thr.idx_build_rle(gw, goff, r)
            print(f"  indexes r=2^{lr} built", flush=True)
    return out


def draw_query(rng, log_rs):
    u = rng.random()
    name = "plain" if u < 0.4 else ("many" if u < 0.8 else "sparse")
    lr = int(rng.choice(log_rs))
    nb = NB_SPARSE if name == "sparse" else NB
    n = int(round(math.exp(rng.uniform(math.log(3), math.log(nb)))))
    n = min(max(n, 3), nb)
    T = int(rng.integers(1, n + 1))
    ids = rng.integers(0, nb, n).astype(np.uint32)
    return name, lr, ids, T


def measure(idx, ids, T, reps, dout):
    """Minimum pass-A ms per variant (nan where a variant does not apply)
    and the result length."""
    times = np.full(len(VARIANTS), np.nan)
    length = 0
    for v, vf in enumerate(thr.VARIANT_FLAGS):
        # the variant the library would run for this flag (ScanCount above
        # 65535 inputs and split above 8 counter bits fall back to carry-save)
        if v and int(thr.select_variants(idx, [(ids, T)], vf)[0]) != v:
            continue
        best = math.inf
        for k in range(reps + 1):
            length = thr.thr_query(idx, ids, T, out=dout, flags=vf | thr.THR_PROFILE)
            if k:
                best = min(best, thr.thr_last_kernel_ms())
        times[v] = best
    return times, length


def collect(indexes, log_rs, count, seed, reps, dout, label):
    rng = np.random.default_rng(seed)
    rows = []
    t0 = time.time()
    while len(rows) < count:
        for attempt in range(20):
            name, lr, ids, T = draw_query(rng, log_rs)
            idx = indexes[(name, lr)]
            # a result of one marker word is empty: draw again
            if thr.thr_query(idx, ids, T, out=dout) > 1 or attempt == 19:
                break
        times, _ = measure(idx, ids, T, reps, dout)
        f = thr.query_features(idx, ids, T)
        rows.append((name, lr, ids, T, f, times))
        if len(rows) % 2000 == 0:
            print(f"  {label}: {len(rows)} queries, {time.time() - t0:.0f} s", flush=True)
    return rows


def rule_design(idx, ids, T):
    words = float(np.sum(idx_lens(idx)[ids]))
    bits = float(np.sum(idx_bits(idx)[ids]))
    n = len(ids)
    S1 = int(T).bit_length()
    S = min(S1, int(n - T + 1).bit_length())
    return words, bits, S, S1


_lens_cache, _bits_cache = {}, {}


def idx_lens(idx):
    return _lens_cache[idx.handle]


def idx_bits(idx):
    return _bits_cache[idx.handle]


def fit_rule(rows, indexes):
    """Least squares fits, times in ms: t = a0 + a1 w + a2 w S (grouped
    carry-save), c0 + c1 w + c2 w S1 (position-major), b0 + b1 w + b2 bits
    (ScanCount), s0 + s1 w + s2 w S (split inputs)."""
    D = [([], []), ([], []), ([], []), ([], [])]
    for name, lr, ids, T, f, times in rows:
        w, bits, S, S1 = rule_design(indexes[(name, lr)], ids, T)
        xs = ([1.0, w, w * S], [1.0, w, w * S1], [1.0, w, bits], [1.0, w, w * S])
        for v in range(4):
            if not math.isnan(times[v]):
                D[v][0].append(xs[v])
                D[v][1].append(times[v])
    out = []
    for A, y in D:
        out += [float(x) for x in np.linalg.lstsq(np.array(A), np.array(y), rcond=None)[0]]
    return out


def totals(times, choice):
    return float(sum(times[i, c] for i, c in enumerate(choice)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="selector_out")
    ap.add_argument("--train", type=int, default=50_000)
    ap.add_argument("--test", type=int, default=5_000)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--epochs", type=int, default=150)
    ap.add_argument("--log-r", type=str, default="18-26")
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    args = ap.parse_args()
    import torch
    torch.cuda.init()
    lo, hi = (int(x) for x in args.log_r.split("-"))
    LOG_R = range(lo, hi + 1)
    t0 = time.time()
    indexes = build_indexes(0, LOG_R, args.workers)
    for idx in indexes.values():
        # per-bitmap compressed words and set rows for the rule's design matrix
        nb = idx.nbitmaps
        n_words = np.zeros(nb)
        n_bits = np.zeros(nb)
        for b in range(nb):
            f = thr.query_features(idx, [b], 1)
            n_words[b] = 2.0 ** f[9] - 1.0
            n_bits[b] = f[15] * idx.r
        _lens_cache[idx.handle] = n_words
        _bits_cache[idx.handle] = n_bits
    print(f"indexes ready in {time.time() - t0:.0f} s", flush=True)
    W_max = (1 << max(LOG_R)) // 64 + 1
    dout = torch.empty(W_max, dtype=torch.int64, device="cuda")

    log_rs = list(LOG_R)
    train = collect(indexes, log_rs, args.train, 1, args.reps, dout, "train")
    test = collect(indexes, log_rs, args.test, 2, args.reps, dout, "held-out")
    print(f"timings collected in {time.time() - t0:.0f} s", flush=True)

    def arrays(rows):
        X = np.stack([r[4] for r in rows]).astype(np.float32)
        Tm = np.stack([r[5] for r in rows])
        M = ~np.isnan(Tm)
        Y = np.where(M, np.log(np.where(M, Tm, 1.0)), 0.0).astype(np.float32)
        return X, Tm, M.astype(np.uint8), Y

    Xtr, Ttr, Mtr, Ytr = arrays(train)
    Xte, Tte, Mte, Yte = arrays(test)
    mean = Xtr.mean(axis=0)
    std = Xtr.std(axis=0)
    istd = np.where(std > 1e-6, 1.0 / np.maximum(std, 1e-6), 0.0).astype(np.float32)
    sel = thr.Selector(seed=0)
    sel.set_norm(mean, istd)
    loss = sel.train(Xtr, Ytr, Mtr, epochs=args.epochs, batch=512, lr=2e-3, seed=3)
    te_loss, _ = sel.gradients(Xte, Yte, Mte)
    print(f"trained: train loss {loss:.4f}, held-out loss {te_loss:.4f} "
          f"({time.time() - t0:.0f} s)", flush=True)

    coeffs = fit_rule(train, indexes)
    thr.rule_model(coeffs)

    # choices on the held-out queries, made by the library's policies
    for idx in indexes.values():
        thr.set_selector(idx, sel)
    learned, rule = [], []
    for name, lr, ids, T, f, times in test:
        ix = indexes[(name, lr)]
        learned.append(int(thr.select_variants(ix, [(ids, T)], thr.THR_POLICY_LEARNED)[0]))
        rule.append(int(thr.select_variants(ix, [(ids, T)], thr.THR_POLICY_RULE)[0]))
    learned, rule = np.array(learned), np.array(rule)
    Tinf = np.where(Mte.astype(bool), Tte, np.inf)
    best = Tinf.argmin(axis=1)
    fixed = np.zeros(len(test), dtype=int)
    single = int(np.argmin([np.sum(np.where(Mte[:, v].astype(bool), Tte[:, v], Tte[:, 0]))
                            for v in range(len(VARIANTS))]))
    single_choice = np.where(Mte[:, single].astype(bool), single, 0)
    res = {
        "queries": {"train": len(train), "held_out": len(test)},
        "reps": args.reps,
        "log_r": [min(LOG_R), max(LOG_R)],
        "loss": {"train": loss, "held_out": te_loss},
        "total_ms": {
            "measured_best": totals(Tinf, best),
            "learned": totals(Tinf, learned),
            "rule": totals(Tinf, rule),
            "fixed_csa": totals(Tinf, fixed),
            "best_single_variant": totals(Tinf, single_choice),
        },
        "agreement_with_best": {
            "learned": float(np.mean(learned == best)),
            "rule": float(np.mean(rule == best)),
            "fixed_csa": float(np.mean(fixed == best)),
        },
        "best_variant_counts": {v: int(np.sum(best == i)) for i, v in enumerate(VARIANTS)},
        "rule_coefficients": coeffs,
        "seconds": round(time.time() - t0, 1),
    }
    tb = res["total_ms"]["measured_best"]
    res["ratio_to_best"] = {k: v / tb for k, v in res["total_ms"].items()}
    print(json.dumps(res, indent=1), flush=True)
    os.makedirs(args.out, exist_ok=True)
    with open(os.path.join(args.out, "selector_weights.json"), "w") as f:
        json.dump({"features": thr.SEL_FEATURES, "variants": list(VARIANTS),
                   "params": [float(x) for x in sel.params()],
                   "mean": [float(x) for x in mean], "istd": [float(x) for x in istd],
                   "rule_coefficients": coeffs}, f)
    with open(os.path.join(args.out, "selector_eval.json"), "w") as f:
        json.dump(res, f, indent=1)
    np.savez_compressed(os.path.join(args.out, "selector_heldout.npz"), X=Xte, times=Tte,
                        mask=Mte, rule=rule, learned=learned)
    for idx in indexes.values():
        idx.close()


if __name__ == "__main__":
    main()
