"""Oracle of the learned cost model -- TEST INFRASTRUCTURE ONLY.

fp64 NumPy forward/backward/Adam of the 3-layer perceptron the tuner trains
on its own timings: inputs (log m, log n, NB/512, IB/256) standardized with
the training set's mean and deviation, two hidden layers of 64 ReLU units,
one linear output predicting log(seconds); loss = mean squared error; Adam
(Kingma & Ba, 2015) with the usual bias correction.

The paper itself argues against models (Secs. 1 and 2.3) and tunes purely
empirically; the model only ranks candidates and the empirical measurement
keeps the final say.

Layout matches the GPU kernels: W1 (64 x 4), W2 (64 x 64), W3 (1 x 64),
row-major [out, in]; y = W x + b per layer.
"""
import numpy as np

LAYERS = [(4, 64), (64, 64), (64, 1)]


def features(m, n, nb, ib):
    """Raw (unstandardized) features of a configuration."""
    return np.array([np.log(m), np.log(n), nb / 512.0, ib / 256.0], dtype=np.float64)


def standardize(X, mean=None, std=None):
    if mean is None:
        mean = X.mean(axis=0)
        std = X.std(axis=0)
        std = np.where(std > 0, std, 1.0)
    return (X - mean) / std, mean, std


def forward(params, X):
    """X: (batch, 4). Returns (yhat (batch,), cache)."""
    W1, b1, W2, b2, W3, b3 = params
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + b3
    return y[:, 0], (X, z1, h1, z2, h2)


def loss(params, X, y):
    yhat, _ = forward(params, X)
    return float(np.mean((yhat - y) ** 2))


def backward(params, cache, yhat, y):
    """Gradients of mean((yhat - y)^2) with respect to every parameter."""
    W1, b1, W2, b2, W3, b3 = params
    X, z1, h1, z2, h2 = cache
    B = X.shape[0]
    dy = (2.0 / B) * (yhat - y)[:, None]          # (B, 1)
    gW3 = dy.T @ h2
    gb3 = dy.sum(axis=0)
    dh2 = dy @ W3
    dz2 = dh2 * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    return [gW1, gb1, gW2, gb2, gW3, gb3]


def adam_step(params, grads, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1). Returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for p, g, mm, vv in zip(params, grads, m, v):
        mm = beta1 * mm + (1 - beta1) * g
        vv = beta2 * vv + (1 - beta2) * g * g
        mh = mm / (1 - beta1 ** t)
        vh = vv / (1 - beta2 ** t)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mm)
        out_v.append(vv)
    return out_p, out_m, out_v


def train(params, X, y, steps, lr=1e-3):
    """Full-batch Adam for `steps` updates. Returns (params, loss history)."""
    m = [np.zeros_like(p) for p in params]
    v = [np.zeros_like(p) for p in params]
    hist = []
    for t in range(1, steps + 1):
        yhat, cache = forward(params, X)
        hist.append(float(np.mean((yhat - y) ** 2)))
        g = backward(params, cache, yhat, y)
        params, m, v = adam_step(params, g, m, v, t, lr)
    return params, hist
