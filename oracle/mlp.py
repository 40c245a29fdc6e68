"""FP64 reference of the learned per-row nnz(C) predictor -- TEST INFRASTRUCTURE ONLY.

The paper's GPU path speeds up the estimate of the output's memory needs
with approximate algorithms (Sec. 5, the optimizations paragraph), and it
sizes batched SpGEMM from a symbolic step (Sec. 7.4, caption of the CA
SpGEMM strong-scaling figure).  The predictor here is that approximate estimator: a
3 -> 64 -> 64 -> 1 MLP over three per-row features of the product.  The paper
fixes none of its details; this file is the plain statement of the reading
used (every step written out in numpy float64):

  features  f_i = (nnz(A(i,:)), flops_i, max_p nnz(B(p,:))), w_i = ncols(B)
  inputs    l_i = (log2(1 + f_i0), log2(1 + f_i1) - log2 w_i, log2(1 + f_i2) - log2 w_i)
            x_i = (l_i - mu) / sigma
            (the last two features relative to the output width, so that one
            network serves products of any size)
  network   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = w3 . h2 + b3
  ratio     rho_i = sigmoid(z_i)             (predicted nnz(C_i) / flops_i)
  size      pred_i = clamp(ceil(rho_i * flops_i), maxB_i, min(flops_i, w_i))
  loss      e_i = log2(nnz_i / flops_i) - log2(rho_i)
            L = mean_i  tau * e_i          if e_i >= 0   (under-prediction)
                        (tau - 1) * e_i    otherwise     (over-prediction)
            over rows with flops_i > 0; tau = 0.9 prefers over-prediction.
  optimiser Adam with bias correction.
"""
from __future__ import annotations

import math

import numpy as np

HIDDEN = 64
LN2 = math.log(2.0)


def init_params(seed: int = 0, hidden: int = HIDDEN) -> dict:
    """He-style random initialisation (any initialisation is valid; this one is seeded)."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.normal(0, math.sqrt(2.0 / 3), (hidden, 3)),
        "b1": np.zeros(hidden),
        "W2": rng.normal(0, math.sqrt(2.0 / hidden), (hidden, hidden)),
        "b2": np.zeros(hidden),
        "w3": rng.normal(0, math.sqrt(1.0 / hidden), (hidden,)),
        "b3": np.zeros(1),
    }


def raw_features(nnz_a, flops, maxb, width) -> np.ndarray:
    """The network's inputs before standardisation (one row per output row)."""
    lw = np.log2(np.maximum(np.asarray(width, dtype=np.float64), 1.0))
    return np.stack([np.log2(1.0 + np.asarray(nnz_a, dtype=np.float64)),
                     np.log2(1.0 + np.asarray(flops, dtype=np.float64)) - lw,
                     np.log2(1.0 + np.asarray(maxb, dtype=np.float64)) - lw], axis=1)


def standardise(F: np.ndarray, mu: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    return (F - mu[None, :]) / sigma[None, :]


def forward(p: dict, X: np.ndarray):
    """Logits z (shape [m]) and the cache needed by backward."""
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["w3"] + p["b3"][0]
    return z, (X, a1, h1, a2, h2)


def log2_sigmoid(z: np.ndarray) -> np.ndarray:
    # log sigmoid(z) = -softplus(-z), written stably.
    return -(np.maximum(-z, 0.0) + np.log1p(np.exp(-np.abs(z)))) / LN2


def sigmoid(z: np.ndarray) -> np.ndarray:
    return np.where(z >= 0, 1.0 / (1.0 + np.exp(-np.abs(z))), np.exp(-np.abs(z)) / (1.0 + np.exp(-np.abs(z))))


def loss_and_dz(z: np.ndarray, flops: np.ndarray, nnz: np.ndarray, tau: float = 0.9):
    """Mean pinball loss over rows with flops > 0 and its gradient with respect to z."""
    flops = np.asarray(flops, dtype=np.float64)
    nnz = np.asarray(nnz, dtype=np.float64)
    live = flops > 0
    cnt = max(int(live.sum()), 1)
    e = np.zeros_like(z)
    e[live] = np.log2(nnz[live] / flops[live]) - log2_sigmoid(z[live])
    L = np.where(e >= 0, tau * e, (tau - 1.0) * e)
    L = np.where(live, L, 0.0).sum() / cnt
    dLde = np.where(e >= 0, tau, tau - 1.0)
    dedz = -(1.0 - sigmoid(z)) / LN2
    dz = np.where(live, dLde * dedz, 0.0) / cnt
    return float(L), dz


def backward(p: dict, cache, dz: np.ndarray) -> dict:
    X, a1, h1, a2, h2 = cache
    g = {"w3": h2.T @ dz, "b3": np.array([dz.sum()])}
    dh2 = np.outer(dz, p["w3"])
    da2 = dh2 * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * (a1 > 0)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(axis=0)
    return g


def predict_sizes(z: np.ndarray, flops, maxb, ncols) -> np.ndarray:
    """Integer per-row size: ceil(sigmoid(z) * flops) clamped to [maxB, min(flops, ncols)]
    (ncols: the output width, one value or one per row)."""
    flops = np.asarray(flops, dtype=np.int64)
    maxb = np.asarray(maxb, dtype=np.int64)
    est = np.ceil(sigmoid(z) * flops.astype(np.float64)).astype(np.int64)
    hi = np.minimum(flops, ncols)
    return np.minimum(np.maximum(est, maxb), hi)


def adam_step(p: dict, g: dict, state: dict, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8) -> None:
    """One Adam update with bias correction (in place); state holds m, v and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1 - beta1) * g[k]
        v[...] = beta2 * v + (1 - beta2) * g[k] * g[k]
        mhat = m / (1 - beta1 ** t)
        vhat = v / (1 - beta2 ** t)
        p[k] = p[k] - lr * mhat / (np.sqrt(vhat) + eps)
