"""The cost model's CUDA kernels (C ABI: qr_mlp_forward / qr_mlp_grad /
qr_mlp_adam_step / qr_mlp_train) against the fp64 oracle of oracle/mlp.py,
whose gradients are pinned by finite differences on the CPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlp
from paper_1102_5328_gb300 import inputs


@pytest.fixture(scope="module")
def cm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1102_5328_gb300 import costmodel
    return costmodel


def _data(n, seed):
    rng = np.random.default_rng(seed)
    Z = rng.standard_normal((n, 4))
    y = np.sin(Z[:, 0]) + 0.3 * Z[:, 1] * Z[:, 2] - 0.5 * Z[:, 3]
    return Z, y


@pytest.mark.parametrize("n", [1, 31, 100, 257])
def test_forward_and_grad_match_oracle(cm, n):
    params = inputs.mlp_init(1)
    Z, y = _data(n, 2)
    model = cm.CostModel(params)
    yh = model.forward(Z)
    yo, cache = mlp.forward(params, Z)
    assert np.allclose(yh, yo, rtol=1e-5, atol=1e-5)
    g, loss = model.grad(Z, y)
    go = cm.flatten(mlp.backward(params, cache, yo, y)).astype(np.float64)
    assert abs(loss - np.mean((yo - y) ** 2)) <= 1e-5 * max(1.0, loss)
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)


def test_adam_step_matches_oracle(cm):
    params = inputs.mlp_init(3)
    Z, y = _data(64, 4)
    model = cm.CostModel(params)
    yo, cache = mlp.forward(params, Z)
    go = mlp.backward(params, cache, yo, y)
    model.adam_step(cm.flatten(go), lr=1e-2)
    zeros = [np.zeros_like(p) for p in params]
    po, _, _ = mlp.adam_step(params, go, zeros, [np.zeros_like(p) for p in params], 1, lr=1e-2)
    assert np.allclose(cm.flatten(model.params()), cm.flatten(po), atol=1e-6)


def test_training_tracks_oracle_and_learns(cm):
    params = inputs.mlp_init(5)
    Z, y = _data(200, 6)
    model = cm.CostModel(params)
    loss_gpu = model.train(Z, y, steps=300, lr=1e-2)
    po, hist = mlp.train(params, Z, y, steps=300, lr=1e-2)
    yg = model.forward(Z)
    yo, _ = mlp.forward(po, Z)
    final_oracle = float(np.mean((yo - y) ** 2))
    assert np.mean((yg - y) ** 2) < 0.3 * hist[0]
    assert abs(np.mean((yg - y) ** 2) - final_oracle) <= 0.05 * hist[0] + 1e-3
    assert loss_gpu > 0
