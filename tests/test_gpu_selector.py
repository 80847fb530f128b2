"""GPU checks of the learned cost model: the CUDA forward and backward passes
against the fp64 oracle of oracle/mlp.py (same BF16-rounded weights, or FP32
weights), training that lowers the loss, the query features against an
independent numpy computation, and the learned policy end to end."""
import numpy as np
import pytest

import oracle
import paper_1402_4466_gb300 as thr
import synth
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()
    return torch


def _data(seed, rows):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((rows, 16)) * 3 + 5).astype(np.float32)
    T = rng.standard_normal((rows, thr.SEL_VARIANTS)).astype(np.float32)
    M = (rng.random((rows, thr.SEL_VARIANTS)) < 0.8).astype(np.uint8)
    mean = X.mean(axis=0).astype(np.float32)
    istd = (1.0 / X.std(axis=0)).astype(np.float32)
    return X, T, M, mean, istd


@pytest.mark.parametrize("fp32,tol", [(False, 1e-4), (True, 1e-5)])
def test_gradients_match_oracle(fp32, tol):
    sel = thr.Selector(seed=3, fp32=fp32)
    X, T, M, mean, istd = _data(1, 300)
    sel.set_norm(mean, istd)
    p = sel.params()
    loss, g = sel.gradients(X, T, M)
    lo, go = mlp.loss_and_grad(p, X, T, M, mean, istd, bf16=not fp32)
    assert loss == pytest.approx(lo, rel=tol)
    scale = np.abs(go).max()
    err = np.abs(g.astype(np.float64) - go).max() / scale
    assert err < tol, f"max gradient error {err:.3g} of the largest gradient"
    # every parameter block receives gradient
    assert np.count_nonzero(g) > 0.9 * g.size


def test_predictions_match_oracle():
    sel = thr.Selector(seed=4)
    X, T, M, mean, istd = _data(2, 1000)
    sel.set_norm(mean, istd)
    y = sel.predict(X)
    yo, _ = mlp.forward(sel.params(), X, mean, istd, bf16=True)
    assert np.abs(y - yo).max() <= 1e-5 * max(1.0, np.abs(yo).max())


def test_training_lowers_the_loss():
    """A smooth target of the features: Adam on the CUDA passes fits it."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((4000, 16)).astype(np.float32)
    w = rng.standard_normal((16, thr.SEL_VARIANTS)).astype(np.float32) * 0.5
    T = np.tanh(X @ w) + 0.3 * (X[:, :thr.SEL_VARIANTS] ** 2)
    M = np.ones_like(T, dtype=np.uint8)
    sel = thr.Selector(seed=6)
    sel.set_norm(np.zeros(16), np.ones(16))
    l0, _ = sel.gradients(X, T, M)
    loss = sel.train(X, T, M, epochs=60, batch=256, lr=3e-3, seed=7)
    l1, _ = sel.gradients(X, T, M)
    assert l1 < 0.05 * l0 and loss < 0.1 * l0, (l0, loss, l1)
    # the trained parameters still give the oracle's outputs
    y = sel.predict(X[:100])
    yo, _ = mlp.forward(sel.params(), X[:100], np.zeros(16), np.ones(16), bf16=True)
    assert np.abs(y - yo).max() <= 1e-5 * max(1.0, np.abs(yo).max())


@pytest.fixture(scope="module")
def small_index():
    r = 300_000
    words, _ = synth.many_criteria(14, 40, r)
    gw, goff = thr.encode_many(words, r)
    ostreams = [oracle.encode(w, r) for w in words]
    return thr.idx_build_rle(gw, goff, r), oracle.Index(ostreams, r), words, gw, goff, r


def test_query_features(small_index):
    g, o, words, gw, goff, r = small_index
    ids = np.array([3, 7, 7, 0, 39, 12], np.uint32)
    T = 2
    f = thr.query_features(g, ids, T)
    lens = np.diff(goff.astype(np.int64))[ids].astype(np.float64)
    dens = np.array([np.unpackbits(words[i].view(np.uint8)).sum() / r for i in ids])
    n = len(ids)
    want = [np.log2(n), np.log2(T + 1), np.log2(n - T + 2), np.log2(r)]
    want += list(np.quantile(np.log2(lens + 1), [0, .25, .5, .75, 1]))
    want += [np.log2(lens.sum() + 1)]
    want += list(np.quantile(np.log10(dens + 1e-7), [0, .25, .5, .75, 1]))
    want += [dens.sum()]
    assert np.allclose(f, np.array(want, np.float32), rtol=1e-6, atol=1e-6)


def test_learned_policy_follows_the_model(small_index):
    g, o, words, gw, goff, r = small_index
    rng = np.random.default_rng(9)
    qs = [(rng.integers(0, 40, int(rng.integers(1, 300))).astype(np.uint32), 0)
          for _ in range(20)]
    qs = [(ids, int(rng.integers(0, len(ids) + 2))) for ids, _ in qs]
    sel = thr.Selector(seed=1)
    p = np.zeros(thr.SEL_PARAMS, np.float32)
    p[-4:] = [1.0, 2.0, -1.0, 3.0]  # W3 = 0: the model predicts ScanCount fastest
    sel.set_params(p)
    thr.set_selector(g, sel)
    try:
        v = thr.select_variants(g, qs, thr.THR_POLICY_LEARNED)
        want = [2] * len(qs)  # ScanCount applies up to 65535 inputs (16-bit counters)
        assert v.tolist() == want
        off, ln, pool = thr.thr_query_batch(g, qs, flags=thr.THR_POLICY_LEARNED)
        for k, (ids, T) in enumerate(qs):
            assert np.array_equal(pool[int(off[k]):int(off[k] + ln[k])], o.threshold(ids, T))
        p[-4:] = [0.0, -1.0, 1.0, 2.0]  # now the position-major decode wins
        sel.set_params(p)
        assert thr.select_variants(g, qs, thr.THR_POLICY_LEARNED).tolist() == [1] * len(qs)
        p[-4:] = [0.0, 1.0, 1.0, -0.05]  # split predicted 5% faster: below the margin
        sel.set_params(p)
        assert thr.select_variants(g, qs, thr.THR_POLICY_LEARNED).tolist() == [0] * len(qs)
        p[-4:] = [0.0, 1.0, 1.0, -1.0]  # split clearly faster (where it applies)
        sel.set_params(p)
        off, ln, pool = thr.thr_query_batch(g, qs, flags=thr.THR_POLICY_LEARNED)
        for k, (ids, T) in enumerate(qs):
            assert np.array_equal(pool[int(off[k]):int(off[k] + ln[k])], o.threshold(ids, T))
    finally:
        thr.set_selector(g, None)
    # without a model the learned policy is the rule chooser
    assert np.array_equal(thr.select_variants(g, qs, thr.THR_POLICY_LEARNED),
                          thr.select_variants(g, qs, thr.THR_POLICY_RULE))


def test_position_variant(small_index):
    g, o, words, gw, goff, r = small_index
    rng = np.random.default_rng(10)
    for n, T in [(30, 29), (40, 38), (200, 190), (5, 5)]:
        ids = rng.integers(0, 40, n).astype(np.uint32)
        got = thr.thr_query(g, ids, T, flags=thr.THR_VARIANT_POSITION)
        assert np.array_equal(got, o.threshold(ids, T))
