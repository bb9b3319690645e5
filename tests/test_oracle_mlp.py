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


def test_growth_targets_by_hand():
    """log1p(max(0, later - then) / horizon): gains 8, 0, -8 (no growth) and
    4 over a horizon of 4 batches are 2, 0, 0 and 1 edges per batch."""
    t = mlp.growth_targets([0, 5, 10, 3], [8, 5, 2, 7], 4.0)
    assert np.allclose(t, [np.log(3.0), 0.0, 0.0, np.log(2.0)], rtol=0, atol=1e-15)
    # swapping the snapshots turns growth into loss, which counts as none
    assert np.allclose(mlp.growth_targets([8, 5, 2, 7], [0, 5, 10, 3], 4.0), [0.0, 0.0, np.log(3.0), 0.0])


def test_adam_first_step_moves_by_the_learning_rate():
    """Adam's first update from zero moments is lr * g / (|g| + eps) after the
    bias corrections cancel (1 - b1) and (1 - b2): a step of lr against the
    gradient's sign wherever |g| >> eps, and none where g = 0."""
    g = np.array([0.5, -2.0, 1e-3, 0.0, 3e-9])
    P, M, V = mlp.adam_step(np.zeros(5), np.zeros(5), np.zeros(5), g, 1, lr=0.01)
    assert np.allclose(P[:2], [-0.01, 0.01], rtol=1e-7, atol=0)
    assert np.isclose(P[2], -0.01 * 1e-3 / (1e-3 + 1e-8), rtol=1e-12)
    assert P[3] == 0.0
    assert np.isclose(P[4], -0.01 * 3e-9 / (3e-9 + 1e-8))
    assert np.allclose(M, 0.1 * g) and np.allclose(V, 0.001 * g * g)


def test_adam_second_step_by_hand():
    """Two steps with gradients 1 then 3 (b1 = 0.9, b2 = 0.999, eps = 0):
    m = 0.1, then 0.39 -> m_hat = 0.39 / 0.19; v = 0.001, then 0.010 ->
    v_hat = 0.010 / 0.001999 (Kingma and Ba, Algorithm 1)."""
    P, M, V = mlp.adam_step(np.array([1.0]), np.zeros(1), np.zeros(1), np.array([1.0]), 1, lr=0.1, eps=0.0)
    assert np.isclose(P[0], 0.9)
    P, M, V = mlp.adam_step(P, M, V, np.array([3.0]), 2, lr=0.1, eps=0.0)
    assert np.isclose(M[0], 0.39) and np.isclose(V[0], 0.999 * 0.001 + 0.001 * 9.0)
    m_hat = 0.39 / (1 - 0.81)
    v_hat = (0.999 * 0.001 + 0.009) / (1 - 0.999 ** 2)
    assert np.isclose(P[0], 0.9 - 0.1 * m_hat / np.sqrt(v_hat))


def test_adam_minimises_a_quadratic():
    """A few hundred steps on f(p) = sum((p - c)^2) bring p to c."""
    c = np.array([3.0, -1.0, 0.25])
    P, M, V = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 2001):
        P, M, V = mlp.adam_step(P, M, V, 2 * (P - c), t, lr=0.05)
    assert np.allclose(P, c, atol=1e-3)
