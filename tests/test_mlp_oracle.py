"""Pins for oracle/mlp.py (CPU only): gradients against central finite
differences, a linear special case in closed form, and Adam's first step."""
import numpy as np
import pytest

from oracle import mlp
from paper_1102_5328_gb300 import inputs


def _data(seed, B=37):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, 4))
    y = rng.standard_normal(B)
    return X, y


@pytest.mark.parametrize("seed", [0, 1])
def test_gradients_match_central_differences(seed):
    params = inputs.mlp_init(seed)
    X, y = _data(seed + 10)
    yhat, cache = mlp.forward(params, X)
    grads = mlp.backward(params, cache, yhat, y)
    h = 1e-6
    worst = 0.0
    for pi, p in enumerate(params):
        flat = p.reshape(-1)
        idxs = range(flat.size) if flat.size <= 64 else np.random.default_rng(pi).choice(flat.size, 64, replace=False)
        for k in idxs:
            old = flat[k]
            flat[k] = old + h
            lp = mlp.loss(params, X, y)
            flat[k] = old - h
            lm = mlp.loss(params, X, y)
            flat[k] = old
            fd = (lp - lm) / (2 * h)
            g = grads[pi].reshape(-1)[k]
            # relative error; gradients below 1e-3 are held to an absolute
            # 1e-9, the size of the difference quotient's rounding error
            worst = max(worst, abs(fd - g) / max(1e-3, abs(fd) + abs(g)))
    assert worst <= 1e-6, worst


def test_linear_special_case_closed_form():
    """With hidden pre-activations kept positive and W2 = I the network is
    affine in its last layer; dL/dW3 = 2/B (yhat - y)^T h2 and dL/db3 =
    2/B sum(yhat - y), written out independently."""
    params = inputs.mlp_init(3)
    params[0] = np.zeros((64, 4))
    params[1] = np.linspace(0.5, 1.5, 64)           # h1 = b1 > 0
    params[2] = np.eye(64)
    params[3] = np.zeros(64)
    X, y = _data(4, B=5)
    yhat, cache = mlp.forward(params, X)
    h2 = np.tile(params[1], (5, 1))
    assert np.allclose(yhat, h2 @ params[4][0] + params[5][0])
    g = mlp.backward(params, cache, yhat, y)
    r = yhat - y
    assert np.allclose(g[4][0], 2.0 / 5 * (r @ h2))
    assert np.isclose(g[5][0], 2.0 / 5 * r.sum())
    # every ReLU is active and W2 = I, so dz1 = dz2 = 2/B r W3 row-wise and
    # dL/dW1 = dz1^T X, dL/db1 = column sums of dz1
    dz = (2.0 / 5 * r)[:, None] * params[4][0][None, :]
    assert np.allclose(g[0], dz.T @ X)
    assert np.allclose(g[1], dz.sum(axis=0))
    assert np.allclose(g[2], dz.T @ h2)


def test_adam_first_step_is_signed_lr():
    params = [np.array([1.0, -2.0, 3.0])]
    grads = [np.array([0.5, -0.25, 0.0])]
    m = [np.zeros(3)]
    v = [np.zeros(3)]
    p, m2, v2 = mlp.adam_step(params, grads, m, v, 1, lr=1e-3)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> lr * g / (|g| + eps)
    assert np.allclose(p[0], [1.0 - 1e-3, -2.0 + 1e-3, 3.0], atol=1e-10)
    assert np.allclose(m2[0], 0.1 * grads[0]) and np.allclose(v2[0], 0.001 * grads[0] ** 2)


def test_training_reduces_loss():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((64, 4))
    y = np.sin(X[:, 0]) + 0.5 * X[:, 1] ** 2 - X[:, 3]
    params, hist = mlp.train(inputs.mlp_init(5), X, y, steps=300, lr=1e-2)
    assert hist[-1] < 0.2 * hist[0]
