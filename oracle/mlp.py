"""FP64 reference for the sketch-size proposal network (test infrastructure only).

The network maps 18 features of a first s = 16 sketch to one of 12 width classes
(class c <-> width 8 * 2^c); it answers the question left open in the paper's
discussion (Sec. 7) of choosing a new r1 from the first run.  Layout of the flat
parameter vector: W1 (128 x 18), b1 (128), W2 (128 x 128), b2 (128), W3 (12 x 128),
b3 (12), row-major.  Weights enter every product rounded to BF16 (round to
nearest even); biases stay as given.  Loss: mean softmax cross-entropy.
Pinned by a central-difference check of the analytic gradient in the tests.
"""
from __future__ import annotations

import numpy as np

IN, H, OUT = 18, 128, 12
SHAPES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (OUT, H)), ("b3", (OUT,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16(w: np.ndarray) -> np.ndarray:
    """Round float32 values to BF16 (nearest even), returned as float64."""
    b = np.asarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


def forward(p: np.ndarray, X: np.ndarray):
    """Logits and the hidden activations for a batch X (count x 18)."""
    q = unpack(p)
    W1, W2, W3 = bf16(q["W1"]), bf16(q["W2"]), bf16(q["W3"])
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1.T + q["b1"], 0.0)
    h2 = np.maximum(h1 @ W2.T + q["b2"], 0.0)
    z = h2 @ W3.T + q["b3"]
    return z, h1, h2


def loss_and_grad(p: np.ndarray, X: np.ndarray, y: np.ndarray):
    """Mean cross-entropy and its gradient (flat, same layout as p); weights
    are treated as their BF16 roundings in every product."""
    q = unpack(p)
    W2, W3 = bf16(q["W2"]), bf16(q["W3"])
    X = np.asarray(X, dtype=np.float64)
    z, h1, h2 = forward(p, X)
    B = X.shape[0]
    zm = z - z.max(axis=1, keepdims=True)
    e = np.exp(zm)
    prob = e / e.sum(axis=1, keepdims=True)
    loss = float(np.mean(-np.log(prob[np.arange(B), y])))
    dz = prob.copy()
    dz[np.arange(B), y] -= 1.0
    dz /= B
    g = {}
    g["W3"] = dz.T @ h2
    g["b3"] = dz.sum(axis=0)
    dh2 = (dz @ W3) * (h2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (h1 > 0)
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(axis=0)
    return loss, pack(g)


def features(sigma16: np.ndarray, eps: float, rows: int, cols: int) -> np.ndarray:
    """The 18 inputs from the 14 trusted scaled sketched singular values at s = 16."""
    s = np.asarray(sigma16, dtype=np.float64)[:14]
    s1 = s[0] if s[0] > 0 else 1e-300
    f = np.empty(18)
    f[:14] = np.log10(np.maximum(s, 1e-30 * s1) / (eps * s1))
    f[14] = np.log10(rows)
    f[15] = np.log10(cols)
    f[16] = np.log10(1.0 / eps)
    f[17] = (f[13] - f[7]) / 6.0
    return f
