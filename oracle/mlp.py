"""CPU oracle for the fitness surrogate -- test infrastructure only.

The surrogate is not in the paper.  It is the small model that pre-screens
EBIC offspring: each series s of columns is summarised by sum-pooled learned
column embeddings and per-column statistics, and a two-hidden-layer MLP
predicts a standardised log-fitness.  This module restates, in float64 numpy,
exactly what the CUDA kernels compute:

    features x (F = 80, zero-padded):
        x[0:64] = sum_{c in s} Emb[c]
        x[64]   = mean_{c in s} colmean[c]
        x[65]   = mean_{c in s} colstd[c]
        x[66]   = |s| / len_scale
    h1 = relu(x W1 + b1)          W1: F x 256
    h2 = relu(h1 W2 + b2)         W2: 256 x 256
    y  = h2 . w3 + b3             w3: 256
    loss = mean_b (y_b - t_b)^2,  t = (log1p(f) - t_mean) / t_std

and the gradients of that loss by hand (reverse mode), plus one Adam step.
Only the test suite imports this module.
"""
from __future__ import annotations

import numpy as np

F = 80
EMB = 64
H = 256


def column_stats(A):
    """Per-column mean and (population) standard deviation of a row-major matrix,
    NaN ignored."""
    A = np.asarray(A, np.float64)
    mean = np.nanmean(A, axis=0)
    std = np.nanstd(A, axis=0)
    return np.nan_to_num(mean), np.nan_to_num(std)


def features(seqs, emb, colmean, colstd, len_scale):
    X = np.zeros((len(seqs), F))
    for b, s in enumerate(seqs):
        s = np.asarray(s)
        X[b, :EMB] = emb[s].sum(0)
        X[b, 64] = colmean[s].mean()
        X[b, 65] = colstd[s].mean()
        X[b, 66] = len(s) / len_scale
    return X


def forward(X, p):
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0)
    y = h2 @ p["w3"] + p["b3"]
    return y, (X, z1, h1, z2, h2)


def loss_and_grads(seqs, t, p, colmean, colstd, len_scale):
    """MSE loss and the gradient of every parameter (Emb, W1, b1, W2, b2, w3, b3)."""
    X = features(seqs, p["Emb"], colmean, colstd, len_scale)
    y, (X, z1, h1, z2, h2) = forward(X, p)
    B = len(seqs)
    loss = np.mean((y - t) ** 2)
    dy = 2.0 * (y - t) / B
    g = {}
    g["w3"] = h2.T @ dy
    g["b3"] = np.array(dy.sum())
    dh2 = np.outer(dy, p["w3"]) * (z2 > 0)
    g["W2"] = h1.T @ dh2
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ p["W2"].T) * (z1 > 0)
    g["W1"] = X.T @ dh1
    g["b1"] = dh1.sum(0)
    dX = dh1 @ p["W1"].T
    gE = np.zeros_like(p["Emb"])
    for b, s in enumerate(seqs):
        for c in s:
            gE[c] += dX[b, :EMB]
    g["Emb"] = gE
    return loss, g


def adam_step(p, g, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, 2015) with bias correction; state keeps m, v, t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    out = {}
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1 - beta1) * g[k]
        v[...] = beta2 * v + (1 - beta2) * g[k] ** 2
        mhat = m / (1 - beta1 ** t)
        vhat = v / (1 - beta2 ** t)
        out[k] = p[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return out


def init_params(C, seed):
    rng = np.random.default_rng(seed)
    return {
        "Emb": rng.standard_normal((C, EMB)) * 0.1,
        "W1": np.vstack([rng.standard_normal((67, H)) * np.sqrt(2.0 / 67), np.zeros((F - 67, H))]),
        "b1": np.zeros(H),
        "W2": rng.standard_normal((H, H)) * np.sqrt(2.0 / H),
        "b2": np.zeros(H),
        "w3": rng.standard_normal(H) * np.sqrt(1.0 / H),
        "b3": np.array(0.0),
    }
