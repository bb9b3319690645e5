"""CPU oracle of the learned-sizing network (TEST INFRASTRUCTURE ONLY).

Plain numpy, float64, written from the definitions and independent of the
CUDA kernels: the 8 -> 64 -> 64 -> 1 ReLU network, its mean-squared-error
loss and the gradient by the chain rule, the per-vertex features and the
bucket rule that turns a prediction into a bucket count.  The parameters are
rounded to bfloat16 (round to nearest even, the rounding of the IEEE
binary32 -> bfloat16 conversion) before use, as the device does; the
gradient is taken with respect to the rounded values.

Parameter layout: W1[8][64], b1[64], W2[64][64], b2[64], W3[64], b3
(4801 values).
"""
from __future__ import annotations

import numpy as np

IN, HID = 8, 64
NPARAMS = IN * HID + HID + HID * HID + HID + HID + 1


def bf16_round(a) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float64.  bfloat16 keeps the top 16 bits of the binary32 pattern."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def unpack(P):
    P = np.asarray(P, dtype=np.float64)
    assert P.shape == (NPARAMS,)
    o = 0
    W1 = P[o:o + IN * HID].reshape(IN, HID); o += IN * HID
    b1 = P[o:o + HID]; o += HID
    W2 = P[o:o + HID * HID].reshape(HID, HID); o += HID * HID
    b2 = P[o:o + HID]; o += HID
    W3 = P[o:o + HID]; o += HID
    b3 = P[o]
    return W1, b1, W2, b2, W3, b3


def forward(P, X, round_bf16=True):
    """Network outputs for the rows of X (n x 8)."""
    Q = bf16_round(P) if round_bf16 else np.asarray(P, np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(Q)
    X = np.asarray(X, np.float64)
    h1 = np.maximum(X @ W1 + b1, 0.0)
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    return h2 @ W3 + b3


def loss(P, X, T, round_bf16=True):
    y = forward(P, X, round_bf16)
    return float(np.mean((y - np.asarray(T, np.float64)) ** 2))


def gradient(P, X, T, round_bf16=True):
    """(dLoss/dP as a flat vector, sum of squared errors)."""
    Q = bf16_round(P) if round_bf16 else np.asarray(P, np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(Q)
    X = np.asarray(X, np.float64)
    T = np.asarray(T, np.float64)
    n = len(X)
    z1 = X @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3 + b3
    e = y - T
    dy = 2.0 * e / n
    gW3 = h2.T @ dy
    gb3 = dy.sum()
    dz2 = np.outer(dy, W3) * (z2 > 0)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2.T) * (z1 > 0)
    gW1 = X.T @ dz1
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return g, float(np.sum(e * e))


def features(hist, in_deg, buckets):
    """V x 8 features from out-degree snapshots hist[k][v] (k batches ago,
    k = 0..4), in-degree and bucket count."""
    hist = np.asarray(hist, np.float64)
    d0 = hist[0]
    lg = lambda x: np.log1p(np.maximum(x, 0.0))  # noqa: E731
    din = np.asarray(in_deg, np.float64)
    b = np.maximum(np.asarray(buckets, np.float64), 1.0)
    cols = [lg(d0)] + [lg(d0 - hist[k]) for k in range(1, 5)] + [lg(din), lg(din) - lg(d0), d0 / (15.0 * b)]
    return np.stack(cols, axis=1)


def learned_buckets(y, deg, horizon, load_factor, max_buckets):
    """clamp(ceil((deg + horizon * expm1(max(y, 0))) / (lf * 15)), 1, max)."""
    growth = np.maximum(np.expm1(np.maximum(np.asarray(y, np.float64), 0.0)), 0.0)
    fut = np.asarray(deg, np.float64) + horizon * growth
    b = np.ceil(fut / (load_factor * 15.0))
    return np.clip(b, 1, max_buckets).astype(np.uint32)


def growth_targets(deg_then, deg_later, horizon):
    """log1p(max(0, later - then) / horizon) per vertex."""
    gain = np.asarray(deg_later, np.float64) - np.asarray(deg_then, np.float64)
    return np.log1p(np.maximum(gain, 0.0) / horizon)


def adam_step(P, M, V, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, "Adam: a method for stochastic
    optimization", ICLR 2015, Algorithm 1) at step t >= 1: biased first and
    second moment estimates, their bias corrections, and the parameter
    step.  Returns (P, M, V)."""
    P, M, V, g = (np.asarray(x, np.float64) for x in (P, M, V, g))
    M = b1 * M + (1.0 - b1) * g
    V = b2 * V + (1.0 - b2) * g * g
    m_hat = M / (1.0 - b1 ** t)
    v_hat = V / (1.0 - b2 ** t)
    return P - lr * m_hat / (np.sqrt(v_hat) + eps), M, V
