"""CPU oracle of the selector's cost model (fp64 numpy).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only tests, smoke() and
the benchmark's CPU legs use it; the library does not import it.

The network maps 16 features to V outputs (one per counting variant; V is
given by the parameter count), 16 -> 64 -> 64 -> V with ReLU on
the two hidden layers:  h1 = relu(W1^T x + b1), h2 = relu(W2^T h1 + b2),
y = W3^T h2 + b3, with x = (features - mean) * istd.  The loss is the mean
of (y - t)^2 over the (row, output) pairs whose mask is set.  Gradients are
those of that loss with respect to the parameter values the forward pass
used: the parameters rounded to bfloat16 (round to nearest, ties to even)
when ``bf16`` is true, else the parameters themselves.  The paper's own
selector is a linear time model per algorithm (Sec. 8.1); this network plays
that role.

Flat parameter layout: W1[16][64] b1[64] W2[64][64] b2[64] W3[64][V] b3[V].

Parity status: pinned by tests/test_oracle_mlp.py (central finite
differences, the linear closed form when every unit is active, and bfloat16
rounding cases worked from the format's definition).
"""
from __future__ import annotations

import numpy as np

F, H, V = 16, 64, 4


def shapes(v: int = V):
    return (("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, v)),
            ("b3", (v,)))


def nparams(v: int = V) -> int:
    return sum(int(np.prod(s)) for _, s in shapes(v))


NPARAMS = nparams()


def outputs_of(size: int) -> int:
    """V of a flat parameter vector of the given size."""
    v = (size - nparams(0)) // (H + 1)
    assert nparams(v) == size, size
    return v


def bf16_round(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even) and return
    them as float64.  bfloat16 keeps the top 16 bits of the float32 pattern;
    rounding adds half an ulp of the dropped part, plus one when the kept
    part is odd (ties to even), and truncates."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    keep_lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + keep_lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params) -> dict:
    p = np.asarray(params, dtype=np.float64)
    out, at = {}, 0
    for name, shape in shapes(outputs_of(p.size)):
        n = int(np.prod(shape))
        out[name] = p[at:at + n].reshape(shape)
        at += n
    return out


def effective(params, bf16: bool) -> np.ndarray:
    """The parameter values the passes use."""
    p = np.asarray(params, dtype=np.float32)
    return bf16_round(p) if bf16 else p.astype(np.float64)


def normalise(X, mean, istd) -> np.ndarray:
    # the library normalises in float32; do the same so inputs agree exactly
    X = np.asarray(X, dtype=np.float32)
    return ((X - np.asarray(mean, np.float32)) * np.asarray(istd, np.float32)).astype(np.float64)


def forward(params, X, mean, istd, bf16: bool = True):
    """Outputs (rows x 3) and the intermediate values."""
    w = unpack(effective(params, bf16))
    x = normalise(X, mean, istd)
    a1 = x @ w["W1"] + w["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w["W2"] + w["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w["W3"] + w["b3"]
    return y, (x, h1, h2)


def loss_and_grad(params, X, T, M, mean, istd, bf16: bool = True):
    """Mean squared error over the masked pairs and its gradient (flat)."""
    w = unpack(effective(params, bf16))
    y, (x, h1, h2) = forward(params, X, mean, istd, bf16)
    m = np.asarray(M, dtype=bool)
    cnt = max(int(m.sum()), 1)
    d = np.where(m, y - np.asarray(T, dtype=np.float32).astype(np.float64), 0.0)
    loss = float((d * d).sum() / cnt)
    dy = 2.0 * d / cnt
    gW3 = h2.T @ dy
    gb3 = dy.sum(axis=0)
    dh2 = (dy @ w["W3"].T) * (h2 > 0)
    gW2 = h1.T @ dh2
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ w["W2"].T) * (h1 > 0)
    gW1 = x.T @ dh1
    gb1 = dh1.sum(axis=0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, grad
