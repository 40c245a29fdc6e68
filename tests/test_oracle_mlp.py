"""Pins of the FP64 predictor reference (oracle/mlp.py).

Gradients are pinned by central finite differences of the loss, the network
by closed forms (zero hidden weights make z = b3 for every row), the loss by
hand-computed pinball values, Adam's first step by its closed form, and the
size rule by its clamp bounds.
"""
import math

import numpy as np
import pytest

from oracle import mlp


def _setup(m=37, seed=3):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(seed)
    for k in p:
        p[k] = p[k] + 0.1 * rng.normal(size=p[k].shape)
    X = rng.normal(size=(m, 3))
    flops = rng.integers(1, 5000, m)
    flops[::9] = 0                                        # rows without products are ignored
    nnz = np.maximum(1, (flops * rng.uniform(0.05, 1.0, m)).astype(np.int64))
    return p, X, flops, nnz


def _loss(p, X, flops, nnz):
    z, _ = mlp.forward(p, X)
    return mlp.loss_and_dz(z, flops, nnz)[0]


def test_gradients_match_finite_differences():
    p, X, flops, nnz = _setup()
    z, cache = mlp.forward(p, X)
    _, dz = mlp.loss_and_dz(z, flops, nnz)
    g = mlp.backward(p, cache, dz)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        idx = np.linspace(0, flat.size - 1, min(flat.size, 12)).astype(int)
        for t in idx:
            old = flat[t]
            flat[t] = old + h
            lp = _loss(p, X, flops, nnz)
            flat[t] = old - h
            lm = _loss(p, X, flops, nnz)
            flat[t] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[t]
            assert abs(fd - an) <= 1e-6 + 1e-5 * abs(fd), (k, t, fd, an)


def test_zero_hidden_layer_gives_constant_logit():
    p, X, flops, nnz = _setup()
    p["w3"][:] = 0.0
    p["b3"][:] = 0.7
    z, cache = mlp.forward(p, X)
    assert np.all(z == 0.7)
    _, dz = mlp.loss_and_dz(z, flops, nnz)
    g = mlp.backward(p, cache, dz)
    assert g["b3"][0] == pytest.approx(dz.sum())
    assert np.all(g["W1"] == 0) and np.all(g["W2"] == 0)       # no signal reaches the hidden layers


def test_pinball_values_by_hand():
    tau = 0.9
    # rho = sigmoid(0) = 1/2; flops 8: under by a factor 2 when nnz = 8, over by 2 when nnz = 2.
    z = np.zeros(2)
    L, dz = mlp.loss_and_dz(z, np.array([8, 8]), np.array([8, 2]), tau)
    # e = log2(1) - log2(1/2) = 1 -> 0.9 ; e = log2(1/4) + 1 = -1 -> 0.1 ; mean 0.5
    assert L == pytest.approx(0.5)
    # de/dz = -(1 - 1/2)/ln2 ; dL/de = 0.9 and -0.1 ; mean over 2 rows
    assert dz[0] == pytest.approx(0.9 * -0.5 / math.log(2) / 2)
    assert dz[1] == pytest.approx(-0.1 * -0.5 / math.log(2) / 2)


def test_adam_first_step_closed_form():
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 1e-3])}
    st = {}
    mlp.adam_step(p, g, st, lr=0.01)
    # after one step m_hat = g and v_hat = g^2, so the step is lr * g / (|g| + eps)
    want = np.array([1.0, -2.0, 0.5]) - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8)
    assert np.allclose(p["w"], want, rtol=0, atol=1e-15)


def test_predicted_sizes_respect_bounds():
    z = np.array([-50.0, 50.0, 0.0, 0.0, 3.0])
    flops = np.array([100, 100, 10, 0, 7])
    maxb = np.array([5, 5, 9, 0, 2])
    s = mlp.predict_sizes(z, flops, maxb, ncols=50)
    assert s.tolist() == [5, 50, 9, 0, 7]         # raise to maxB, cap at ncols, raise to maxB, empty, ceil


def test_sigmoid_and_log_sigmoid_are_stable():
    z = np.array([-800.0, -30.0, 0.0, 30.0, 800.0])
    s = mlp.sigmoid(z)
    assert np.all(np.isfinite(s)) and s[2] == 0.5
    ls = mlp.log2_sigmoid(z)
    assert np.all(np.isfinite(ls))
    assert ls[0] == pytest.approx(-800.0 / math.log(2))
