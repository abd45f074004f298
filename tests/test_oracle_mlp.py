"""Pins for the surrogate's CPU oracle (oracle/mlp.py).

The surrogate is not part of the paper, so the pins come from mathematics:
central finite differences of the loss (independent of the hand-written
reverse pass), features of hand-built series, the closed form of Adam's first
step and its convergence on a quadratic, and column statistics of a matrix
small enough to compute by hand.
"""
import numpy as np
import pytest

from oracle import mlp


def _setup(C=12, B=6, seed=3):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(C, seed)
    # non-zero biases and padded W1 rows so that every term of the reverse pass
    # is exercised (the init leaves them zero)
    p["b1"] = rng.standard_normal(mlp.H) * 0.1
    p["b2"] = rng.standard_normal(mlp.H) * 0.1
    p["b3"] = np.array(0.3)
    p["W1"][67:] = rng.standard_normal((mlp.F - 67, mlp.H)) * 0.05
    seqs = [rng.choice(C, size=int(rng.integers(2, 7)), replace=False) for _ in range(B)]
    colmean = rng.standard_normal(C)
    colstd = rng.uniform(0.5, 2.0, C)
    t = rng.standard_normal(B)
    return p, seqs, colmean, colstd, t


def test_features_hand():
    C = 5
    emb = np.arange(C * mlp.EMB, dtype=np.float64).reshape(C, mlp.EMB) / 100.0
    colmean = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    colstd = np.array([0.5, 0.25, 1.0, 2.0, 4.0])
    X = mlp.features([[4, 0, 2]], emb, colmean, colstd, len_scale=8)
    assert X.shape == (1, 80)
    np.testing.assert_allclose(X[0, :64], emb[4] + emb[0] + emb[2], rtol=0, atol=1e-15)
    assert X[0, 64] == pytest.approx((5 + 1 + 3) / 3, abs=1e-15)
    assert X[0, 65] == pytest.approx((4.0 + 0.5 + 1.0) / 3, abs=1e-15)
    assert X[0, 66] == 3 / 8
    assert np.all(X[0, 67:] == 0)


def test_features_order_invariant():
    """Sum pooling: a series and its reversal have the same features."""
    p, seqs, cm, cs, _ = _setup()
    a = mlp.features(seqs, p["Emb"], cm, cs, 16)
    b = mlp.features([s[::-1] for s in seqs], p["Emb"], cm, cs, 16)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)


def test_gradients_match_finite_differences():
    p, seqs, cm, cs, t = _setup()
    _, g = mlp.loss_and_grads(seqs, t, p, cm, cs, 16)
    rng = np.random.default_rng(11)
    h = 1e-6
    used_cols = sorted({int(c) for s in seqs for c in s})
    for name in ["Emb", "W1", "b1", "W2", "b2", "w3", "b3"]:
        arr = p[name]
        if arr.ndim == 0:
            picks = [()]
        elif name == "Emb":
            picks = [(int(rng.choice(used_cols)), int(rng.integers(mlp.EMB))) for _ in range(24)]
            picks.append((next(c for c in range(12) if c not in used_cols) if len(used_cols) < 12 else used_cols[0], 0))
        else:
            picks = [tuple(int(rng.integers(n)) for n in arr.shape) for _ in range(24)]
        for ix in picks:
            q = {k: v.copy() for k, v in p.items()}
            q[name][ix] += h
            lp, _ = mlp.loss_and_grads(seqs, t, q, cm, cs, 16)
            q[name][ix] -= 2 * h
            lm, _ = mlp.loss_and_grads(seqs, t, q, cm, cs, 16)
            fd = (lp - lm) / (2 * h)
            an = g[name][ix]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, ix, fd, an)


def test_unused_embedding_rows_get_no_gradient():
    p, seqs, cm, cs, t = _setup()
    _, g = mlp.loss_and_grads(seqs, t, p, cm, cs, 16)
    used = {int(c) for s in seqs for c in s}
    for c in range(p["Emb"].shape[0]):
        if c not in used:
            assert np.all(g["Emb"][c] == 0)


def test_loss_is_mean_squared_error_of_forward():
    p, seqs, cm, cs, t = _setup()
    X = mlp.features(seqs, p["Emb"], cm, cs, 16)
    y, _ = mlp.forward(X, p)
    loss, _ = mlp.loss_and_grads(seqs, t, p, cm, cs, 16)
    assert loss == pytest.approx(float(np.mean((y - t) ** 2)), rel=1e-14)
    # a single hidden unit path by hand: zero all weights but one
    q = {k: np.zeros_like(v) for k, v in p.items()}
    q["W1"][66, 5] = 2.0      # h1[5] = 2 * |s| / len_scale
    q["W2"][5, 7] = 3.0       # h2[7] = 3 * h1[5]
    q["w3"][7] = 0.5
    q["b3"] = np.array(-1.0)
    y, _ = mlp.forward(mlp.features([[0, 1, 2, 3]], q["Emb"], cm, cs, 16), q)
    assert y[0] == pytest.approx(0.5 * 3.0 * 2.0 * 4 / 16 - 1.0, abs=1e-15)


def test_adam_first_step_closed_form():
    """With zero moments, bias correction makes the first step -lr g / (|g| + eps)."""
    p = {"a": np.array([1.0, -2.0, 3.0, 0.5])}
    g = {"a": np.array([0.3, -4.0, 1e-3, 0.0])}
    out = mlp.adam_step(p, g, {}, lr=0.01)
    ga = g["a"]
    expect = p["a"] - 0.01 * ga / (np.abs(ga) + 1e-8)
    np.testing.assert_allclose(out["a"], expect, rtol=0, atol=1e-12)


def test_adam_minimises_a_quadratic():
    target = np.array([3.0, -1.5, 0.25])
    p = {"a": np.zeros(3)}
    st = {}
    for _ in range(3000):
        g = {"a": 2.0 * (p["a"] - target)}
        p = mlp.adam_step(p, g, st, lr=0.01)
    np.testing.assert_allclose(p["a"], target, atol=1e-3)


def test_column_stats_hand():
    A = np.array([[1.0, 4.0], [3.0, np.nan], [5.0, 8.0]])
    m, s = mlp.column_stats(A)
    np.testing.assert_allclose(m, [3.0, 6.0], atol=1e-15)
    np.testing.assert_allclose(s, [np.sqrt(8.0 / 3.0), 2.0], atol=1e-15)


def test_training_reduces_loss():
    """Plain gradient steps on the oracle's own gradients reduce the loss."""
    p, seqs, cm, cs, t = _setup(B=16)
    l0, _ = mlp.loss_and_grads(seqs, t, p, cm, cs, 16)
    st = {}
    for _ in range(40):
        _, g = mlp.loss_and_grads(seqs, t, p, cm, cs, 16)
        p = mlp.adam_step(p, g, st, lr=1e-3)
    l1, _ = mlp.loss_and_grads(seqs, t, p, cm, cs, 16)
    assert l1 < 0.5 * l0
