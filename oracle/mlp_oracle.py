"""FP64 CPU reference of the T0-predictor network (test infrastructure only).

The network maps 6 features to 2 outputs: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2),
y = W3 h2 + b3 (128 hidden units), loss = mean over rows and outputs of (y - t)^2. The
parameter vector is flat: W1[128][6], b1[128], W2[128][128], b2[128], W3[2][128], b3[2].
Forward and backward are written out with numpy matrix products (one per step); the
gradient is pinned by central finite differences in the tests. Only tests/ may import it.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 6, 128, 2
SIZES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def forward(p: np.ndarray, x: np.ndarray):
    w = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.tanh(x @ w["W1"].T + w["b1"])
    h2 = np.tanh(h1 @ w["W2"].T + w["b2"])
    y = h2 @ w["W3"].T + w["b3"]
    return y, (x, h1, h2)


def loss_and_grad(p: np.ndarray, x: np.ndarray, t: np.ndarray):
    """loss = sum (y - t)^2 / (rows * 2) and its gradient with respect to p."""
    w = unpack(p)
    y, (x, h1, h2) = forward(p, x)
    rows = x.shape[0]
    d = y - np.asarray(t, dtype=np.float64)
    loss = float(np.sum(d * d) / (rows * N_OUT))
    gy = 2.0 * d / (rows * N_OUT)
    g = {}
    g["W3"] = gy.T @ h2
    g["b3"] = gy.sum(axis=0)
    ga2 = (gy @ w["W3"]) * (1.0 - h2 * h2)
    g["W2"] = ga2.T @ h1
    g["b2"] = ga2.sum(axis=0)
    ga1 = (ga2 @ w["W2"]) * (1.0 - h1 * h1)
    g["W1"] = ga1.T @ x
    g["b1"] = ga1.sum(axis=0)
    return loss, pack(g)
