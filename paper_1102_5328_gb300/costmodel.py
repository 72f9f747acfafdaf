"""Python binding of the tuner's MLP cost model (kernels in tileqr_mlp.cu).

Marshalling only: features are standardized here (mean/deviation of the
training set), every forward/backward/Adam step runs in the CUDA library."""
import ctypes

import numpy as np
import torch

from . import _lib, lib

NPARAMS = 4545


def features(m, n, nb, ib):
    """Raw features (log m, log n, NB/512, IB/256) for arrays of configurations."""
    m, n, nb, ib = (np.asarray(v, dtype=np.float64) for v in (m, n, nb, ib))
    return np.stack([np.log(m), np.log(n), nb / 512.0, ib / 256.0], axis=1)


def flatten(params):
    """[W1, b1, W2, b2, W3, b3] -> flat float32 vector of the kernels' layout."""
    return np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1) for p in params]).astype(np.float32)


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


class CostModel:
    def __init__(self, init_params, device="cuda"):
        self.dev = device
        self.P = torch.from_numpy(flatten(init_params)).to(device)
        assert self.P.numel() == NPARAMS
        self.m = torch.zeros(NPARAMS, dtype=torch.float32, device=device)
        self.v = torch.zeros(NPARAMS, dtype=torch.float32, device=device)
        self.t = 0
        self.mean = None
        self.std = None

    def standardize(self, F, fit=False):
        if fit or self.mean is None:
            self.mean = F.mean(axis=0)
            sd = F.std(axis=0)
            self.std = np.where(sd > 0, sd, 1.0)
        return (F - self.mean) / self.std

    def _x(self, Z):
        return torch.from_numpy(np.ascontiguousarray(Z, dtype=np.float32)).to(self.dev)

    def forward(self, Z):
        X = self._x(Z)
        out = torch.empty(X.shape[0], dtype=torch.float32, device=self.dev)
        _lib.check(lib().qr_mlp_forward(X.shape[0], _p(X), _p(self.P), _p(out), None), "qr_mlp_forward")
        return out.cpu().numpy().astype(np.float64)

    def grad(self, Z, y):
        X = self._x(Z)
        Y = torch.from_numpy(np.asarray(y, dtype=np.float32)).to(self.dev)
        w = ctypes.c_int64()
        lib().qr_mlp_workspace(X.shape[0], ctypes.byref(w))
        work = torch.empty(w.value, dtype=torch.float32, device=self.dev)
        g = torch.empty(NPARAMS + 1, dtype=torch.float32, device=self.dev)
        _lib.check(lib().qr_mlp_grad(X.shape[0], _p(X), _p(Y), _p(self.P), _p(g), _p(work), None), "qr_mlp_grad")
        g = g.cpu().numpy().astype(np.float64)
        return g[:NPARAMS], g[NPARAMS]

    def adam_step(self, grads, lr=1e-3):
        self.t += 1
        G = torch.from_numpy(np.asarray(grads, dtype=np.float32)).to(self.dev)
        _lib.check(lib().qr_mlp_adam_step(_p(G), _p(self.P), _p(self.m), _p(self.v), self.t, lr, None),
                   "qr_mlp_adam_step")

    def train(self, Z, y, steps, lr=1e-3):
        X = self._x(Z)
        Y = torch.from_numpy(np.asarray(y, dtype=np.float32)).to(self.dev)
        w = ctypes.c_int64()
        lib().qr_mlp_workspace(X.shape[0], ctypes.byref(w))
        work = torch.empty(w.value, dtype=torch.float32, device=self.dev)
        g = torch.empty(NPARAMS + 1, dtype=torch.float32, device=self.dev)
        if self.t:
            raise RuntimeError("train() starts Adam at step 1; use a fresh model")
        _lib.check(lib().qr_mlp_train(X.shape[0], _p(X), _p(Y), _p(self.P), _p(self.m), _p(self.v), steps, lr, _p(g),
                                      _p(work), None), "qr_mlp_train")
        self.t = steps
        return float(g[NPARAMS].item())

    def params(self):
        p = self.P.cpu().numpy().astype(np.float64)
        return [p[0:256].reshape(64, 4), p[256:320], p[320:4416].reshape(64, 64), p[4416:4480], p[4480:4544].reshape(1, 64),
                p[4544:4545]]
