"""GPU least squares (C ABI: qr_solve_ls) against the oracle's refined
reference solution: FP64 QR solve and the FP32-factor + FP64-refinement
mixed solve, on conditioned problems with large residuals."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1102_5328_gb300 import inputs

U = 2.0 ** -53


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1102_5328_gb300 as q
    q.lib()
    return q


def to_dev(x):
    x = np.asarray(x)
    if x.ndim == 1:
        x = x[:, None]
    return torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()


def fwd_err(X, Xref):
    return np.linalg.norm(X - Xref, axis=0) / np.linalg.norm(Xref, axis=0)


def test_consistent_system(q):
    A = inputs.uniform_matrix(500, 200, seed=1)
    x0 = inputs.normal_matrix(200, 2, seed=2)
    B = A @ x0
    for prec, it in [(q.QR_PREC_F64, 0), (q.QR_PREC_F32, 30)]:
        X, info = q.qr_solve_ls(to_dev(A), to_dev(B), prec=prec, nb=64, ib=16, max_iter=it)
        err = fwd_err(X.cpu().numpy(), x0).max()
        assert err < 1e3 * U * np.linalg.cond(A), (prec, err)
        assert info[1] in (1, 2) and info[2] == 0


@pytest.mark.parametrize("m,n,kappa,nb,ib", [(600, 200, 1e5, 64, 16), (1024, 512, 1e6, 128, 32),
                                             (777, 300, 1e4, 96, 24)])
def test_mixed_matches_fp64_forward_error(q, m, n, kappa, nb, ib):
    """Large-residual problems (b ~ N(0,1)): the mixed solve refined in FP64
    reaches the FP64 QR solve's forward error (within 2x) against the
    oracle's doubled-precision refined solution."""
    A, B = inputs.ls_problem(m, n, 3, kappa=kappa, seed=int(kappa) % 97 + m)
    Xref, _ = oracle.ls_refine(A, B, maxit=30)
    X64, info64 = q.qr_solve_ls(to_dev(A), to_dev(B), prec=q.QR_PREC_F64, nb=nb, ib=ib)
    Xmx, infomx = q.qr_solve_ls(to_dev(A), to_dev(B), prec=q.QR_PREC_F32, nb=nb, ib=ib, max_iter=50)
    e64 = fwd_err(X64.cpu().numpy(), Xref)
    emx = fwd_err(Xmx.cpu().numpy(), Xref)
    assert infomx[1] in (1, 2), infomx  # tolerance met, or limiting accuracy reached
    assert np.all(emx <= 2 * e64 + 1e3 * U * kappa), (emx, e64)
    # FP64 path: within the LS perturbation bound kappa u + kappa^2 u tan(theta)
    assert np.all(e64 <= 50 * n * U * kappa * (1 + kappa)), e64


def _normal_eq(A, B, X):
    R = B - A @ X
    return np.linalg.norm(A.T @ R, axis=0) / (np.linalg.norm(A, 2) * np.linalg.norm(R, axis=0))


def test_normal_equations_residual(q):
    """||A^T r|| / (||A|| ||r||) of the mixed solution is as small as that of
    the oracle's reference solution, up to the fp64 evaluation noise of the
    check itself (of order kappa u)."""
    kappa = 1e6
    A, B = inputs.ls_problem(2048, 512, 4, kappa=kappa, seed=5)
    X, info = q.qr_solve_ls(to_dev(A), to_dev(B), prec=q.QR_PREC_F32, nb=128, ib=32, max_iter=50)
    Xref, _ = oracle.ls_refine(A, B, maxit=30)
    ne = _normal_eq(A, B, X.cpu().numpy())
    ne_ref = _normal_eq(A, B, Xref)
    assert np.all(ne <= 4 * ne_ref + 10 * kappa * U), (ne, ne_ref)


@pytest.mark.parametrize("m,n,nrhs,p", [(100, 40, 1, 1), (700, 130, 10, 1), (3000, 1100, 9, 4), (5000, 64, 3, 8)])
def test_plain_solve_shapes(q, m, n, nrhs, p):
    """Plain FP64 solve against the oracle's QR solve: one row block of the
    triangular solves (n < 64), ragged last blocks (130 = 2 x 64 + 2,
    1100 = 17 x 64 + 12), an exact multiple, and several groups of <= 8
    right-hand sides."""
    A = inputs.uniform_matrix(m, n, seed=m + n)
    B = inputs.normal_matrix(m, nrhs, seed=nrhs)
    Xo = oracle.ls_solve(A, B)
    X, info = q.qr_solve_ls(to_dev(A), to_dev(B), prec=q.QR_PREC_F64, nb=64, ib=8, p=p)
    assert info[2] == 0
    err = fwd_err(X.cpu().numpy(), Xo)
    kappa = np.linalg.cond(A)
    assert np.all(err < 1e3 * n * U * kappa * (1 + kappa)), err
