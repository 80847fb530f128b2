"""What the trained cost model gains over the method without it, on the
held-out queries of the selector workload (5000 queries drawn like the
training set; per counting variant the minimum of 5 measured pass-A times on
a GB300, stored in tests/data/selector_heldout.npz by train_selector).

The shipped model (paper_1402_4466_gb300/selector_weights.json) is evaluated
with the fp64 oracle of the network on the stored features, so this runs on
the CPU: its choices must cost no more total time than the rule chooser's
(the paper's time-model choice, refit on the same timings) and must agree
with the measured best variant at least as often."""
import json
import os

import numpy as np

from oracle import mlp

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(os.path.dirname(HERE), "paper_1402_4466_gb300", "selector_weights.json")


def _load():
    d = np.load(os.path.join(HERE, "data", "selector_heldout.npz"))
    with open(WEIGHTS) as f:
        w = json.load(f)
    return d, w


def test_learned_choice_beats_the_rule_on_held_out_queries():
    d, w = _load()
    X, times, mask, rule = d["X"], d["times"], d["mask"].astype(bool), d["rule"]
    y, _ = mlp.forward(np.asarray(w["params"], np.float32), X, w["mean"], w["istd"], bf16=True)
    # the learned policy: the fastest predicted variant, but another than the
    # default (0) only when predicted at least 10% faster
    yy = np.where(mask, y, np.inf)
    yy[:, 0] -= np.log(1.1)
    learned = yy.argmin(axis=1)
    if "learned" in d:  # the library's own choices on the same queries
        assert np.mean(learned == d["learned"]) > 0.99
    t = np.where(mask, times, np.inf)
    best = t.argmin(axis=1)
    rows = np.arange(len(t))
    total = {"best": t[rows, best].sum(), "learned": t[rows, learned].sum(),
             "rule": t[rows, rule].sum(), "fixed": t[rows, 0].sum()}
    assert np.isfinite(total["learned"]) and np.isfinite(total["rule"])
    assert total["learned"] <= total["rule"], total
    assert total["learned"] <= total["fixed"], total
    assert np.mean(learned == best) >= np.mean(rule == best)
    # the model's predictions of log time are close on held-out queries
    err = np.where(mask, y - np.log(np.where(mask, times, 1.0)), 0.0)
    assert np.sqrt((err ** 2).sum() / mask.sum()) < 0.1
