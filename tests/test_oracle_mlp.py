"""Pins for the learned-sizing oracle: the analytic gradient against central
finite differences of the loss (which never touches the backward code), a
closed-form case, the bfloat16 rounding against known bit patterns, and the
features and bucket rule on hand-computed values."""
import numpy as np

from oracle import mlp


def test_bf16_rounding_known_patterns():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7 + 2 ** -9, -3.140625, 65504.0, 1.0 + 2 ** -7 + 3 * 2 ** -9,
                     1.0 + 3 * 2 ** -8], np.float32)
    r = mlp.bf16_round(vals)
    # 1 + 2^-8 is exactly halfway between 1 and 1 + 2^-7: ties go to even (1.0)
    assert r[0] == 1.0 and r[1] == 1.0
    assert r[2] == 1.0 + 2 ** -7            # nearer the lower neighbour
    assert r[5] == 1.0 + 2 ** -6            # nearer the upper neighbour
    assert r[6] == 1.0 + 2 ** -6            # halfway between 1 + 2^-7 (odd) and 1 + 2^-6 (even): to even
    assert r[3] == -3.140625
    assert r[4] == 65536.0
    # every result is representable: its low 16 bits are zero
    bits = r.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    P = rng.normal(0, 0.3, mlp.NPARAMS)
    X = rng.normal(0, 1, (40, 8))
    T = rng.normal(0, 1, 40)
    g, sse = mlp.gradient(P, X, T, round_bf16=False)
    assert np.isclose(sse / 40, mlp.loss(P, X, T, round_bf16=False))
    idx = rng.choice(mlp.NPARAMS, 120, replace=False)
    idx = np.concatenate([idx, [mlp.NPARAMS - 1, 0, 8 * 64 + 3]])
    h = 1e-6
    for i in idx:
        Pp = P.copy(); Pp[i] += h
        Pm = P.copy(); Pm[i] -= h
        fd = (mlp.loss(Pp, X, T, False) - mlp.loss(Pm, X, T, False)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_linear_regime_closed_form():
    """With W1 = [I | 0], b1 = 1 (so layer 1 passes x + 1 for x > -1),
    W2 = I and W3 = w, the network is y = w . (x + 1) + b3 on the first
    8 units, and the gradient with respect to W3 is the least-squares one."""
    W1 = np.zeros((8, 64)); W1[:, :8] = np.eye(8)
    b1 = np.zeros(64); b1[:8] = 1.0
    W2 = np.eye(64)
    b2 = np.zeros(64)
    w = np.arange(64) / 64.0
    P = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w, [0.5]])
    rng = np.random.default_rng(1)
    X = rng.uniform(-0.5, 0.5, (30, 8))
    T = rng.normal(0, 1, 30)
    y = mlp.forward(P, X, round_bf16=False)
    assert np.allclose(y, (X + 1.0) @ w[:8] + 0.5)
    g, _ = mlp.gradient(P, X, T, round_bf16=False)
    gW3 = g[8 * 64 + 64 + 64 * 64 + 64: 8 * 64 + 64 + 64 * 64 + 64 + 64]
    e = y - T
    assert np.allclose(gW3[:8], 2.0 / 30 * (X + 1.0).T @ e)
    assert np.allclose(gW3[8:], 0.0)


def test_features_and_bucket_rule_by_hand():
    hist = np.array([[10, 0, 3], [8, 0, 3], [5, 0, 1], [5, 0, 0], [2, 0, 0]])
    X = mlp.features(hist, in_deg=[4, 0, 7], buckets=[1, 1, 2])
    assert np.isclose(X[0, 0], np.log1p(10)) and np.isclose(X[0, 1], np.log1p(2)) and np.isclose(X[0, 4], np.log1p(8))
    assert np.isclose(X[0, 6], np.log1p(4) - np.log1p(10)) and np.isclose(X[0, 7], 10 / 15)
    assert np.allclose(X[1], 0.0)
    assert np.isclose(X[2, 7], 3 / 30)
    # y = log1p(2) -> 2 edges per batch; 10 + 8 * 2 = 26 -> ceil(26 / 10.5) = 3
    b = mlp.learned_buckets([np.log1p(2.0), -1.0, 0.0], [10, 0, 100], 8, 0.7, 1000)
    assert b.tolist() == [3, 1, 10]
    assert mlp.learned_buckets([50.0], [0], 8, 0.7, 7).tolist() == [7]
