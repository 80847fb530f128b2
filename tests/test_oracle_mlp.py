"""Pins of the cost-model oracle (oracle/mlp.py) against facts that do not
come from the oracle itself: central finite differences of its loss, the
linear closed form the network reduces to when every hidden unit is active,
and bfloat16 rounding worked out from the format (8 significant bits, round
to nearest, ties to even)."""
import numpy as np
import pytest

from oracle import mlp


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(mlp.NPARAMS) * scale).astype(np.float32)


def _data(seed, rows=7):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((rows, mlp.F)).astype(np.float32)
    T = rng.standard_normal((rows, mlp.V)).astype(np.float32)
    M = rng.random((rows, mlp.V)) < 0.7
    mean = rng.standard_normal(mlp.F).astype(np.float32) * 0.1
    istd = (1.0 + rng.random(mlp.F)).astype(np.float32)
    return X, T, M, mean, istd


def test_bf16_rounding_cases():
    # representable values are unchanged
    assert mlp.bf16_round([1.0, -2.0, 0.5, 1.0 + 2 ** -7])[3] == 1.0 + 2 ** -7
    # half-way cases go to the even significand
    assert mlp.bf16_round([1.0 + 2 ** -8])[0] == 1.0
    assert mlp.bf16_round([1.0 + 3 * 2 ** -8])[0] == 1.0 + 2 ** -6
    # above half-way rounds up, below rounds down
    assert mlp.bf16_round([1.0 + 2 ** -8 + 2 ** -20])[0] == 1.0 + 2 ** -7
    assert mlp.bf16_round([1.0 + 2 ** -8 - 2 ** -20])[0] == 1.0
    # negative values round symmetrically
    assert mlp.bf16_round([-(1.0 + 3 * 2 ** -8)])[0] == -(1.0 + 2 ** -6)
    # round to nearest with 8 significant bits: relative error <= 2^-8
    # (unit roundoff); truncation would reach 2^-7
    x = np.random.default_rng(0).standard_normal(1000).astype(np.float32)
    r = mlp.bf16_round(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8)


def test_gradient_matches_central_differences():
    p = _params(1).astype(np.float64)
    X, T, M, mean, istd = _data(2)
    loss, g = mlp.loss_and_grad(p, X, T, M, mean, istd, bf16=False)
    rng = np.random.default_rng(3)
    # fp32 parameters: perturb in float64 through a float64 forward
    def f(q):
        w = mlp.unpack(q)
        x = mlp.normalise(X, mean, istd)
        h1 = np.maximum(x @ w["W1"] + w["b1"], 0)
        h2 = np.maximum(h1 @ w["W2"] + w["b2"], 0)
        y = h2 @ w["W3"] + w["b3"]
        d = np.where(M, y - T.astype(np.float64), 0.0)
        return (d * d).sum() / M.sum()
    assert abs(f(p) - loss) < 1e-9 * max(1.0, abs(loss))
    idx = rng.choice(mlp.NPARAMS, 60, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = 1e-6
        fd = (f(p + e) - f(p - e)) / 2e-6
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(fd)), (i, fd, g[i])


def test_linear_closed_form_when_all_units_active():
    """Positive inputs and weights keep every ReLU active: the network is the
    product of its affine maps, written out here as one matrix."""
    rng = np.random.default_rng(4)
    p = np.abs(rng.standard_normal(mlp.NPARAMS)).astype(np.float32) * 0.1
    X = np.abs(rng.standard_normal((5, mlp.F))).astype(np.float32)
    mean = np.zeros(mlp.F, np.float32)
    istd = np.ones(mlp.F, np.float32)
    y, _ = mlp.forward(p, X, mean, istd, bf16=False)
    w = mlp.unpack(p.astype(np.float64))
    A = w["W1"] @ w["W2"] @ w["W3"]                       # 16 x 3
    c = (w["b1"] @ w["W2"] + w["b2"]) @ w["W3"] + w["b3"]  # 3
    assert np.allclose(y, X.astype(np.float64) @ A + c, rtol=1e-12, atol=1e-12)


def test_masked_pairs_do_not_count():
    p = _params(5)
    X, T, M, mean, istd = _data(6)
    T2 = T.copy()
    T2[~M] += 100.0
    l1, g1 = mlp.loss_and_grad(p, X, T, M, mean, istd)
    l2, g2 = mlp.loss_and_grad(p, X, T2, M, mean, istd)
    assert l1 == l2 and np.array_equal(g1, g2)


def test_bf16_gradient_is_taken_at_the_rounded_values():
    p = _params(7)
    X, T, M, mean, istd = _data(8)
    lb, gb = mlp.loss_and_grad(p, X, T, M, mean, istd, bf16=True)
    lr, gr = mlp.loss_and_grad(mlp.bf16_round(p), X, T, M, mean, istd, bf16=False)
    assert lb == pytest.approx(lr, rel=1e-15) and np.allclose(gb, gr, rtol=1e-15, atol=0)
