"""The trained cost model of the variant selector, as shipped with the
package (selector_weights.json, written by ``train_selector`` from timings
measured on a GB300), and the rule chooser's coefficients fitted on the same
timings.

    from paper_1402_4466_gb300 import selector_weights
    sel = selector_weights.attach(idx)   # THR_POLICY_LEARNED now uses it
"""
from __future__ import annotations

import json
import os

import numpy as np

import paper_1402_4466_gb300 as thr

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights.json")


def load(path: str = PATH) -> dict:
    with open(path) as f:
        d = json.load(f)
    if len(d["params"]) != thr.SEL_PARAMS or len(d.get("rule_coefficients", [])) not in (0, 12):
        raise ValueError(f"{path}: written for another library version "
                         f"({len(d['params'])} parameters, {thr.SEL_PARAMS} expected); "
                         "retrain with train_selector")
    return d


def make_selector(path: str = PATH) -> "thr.Selector":
    d = load(path)
    sel = thr.Selector(seed=0)
    sel.set_params(np.asarray(d["params"], np.float32))
    sel.set_norm(np.asarray(d["mean"], np.float32), np.asarray(d["istd"], np.float32))
    return sel


def attach(idx: "thr.Index", path: str = PATH, rule: bool = True) -> "thr.Selector":
    """Attach the shipped model to idx (and set the fitted rule
    coefficients, which THR_POLICY_RULE uses); returns the selector, which
    stays attached while the index lives."""
    d = load(path)
    if rule and "rule_coefficients" in d:
        thr.rule_model(d["rule_coefficients"])
    sel = make_selector(path)
    thr.set_selector(idx, sel)
    return sel
