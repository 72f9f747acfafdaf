"""GPU least squares (C ABI: qr_solve_ls) against the oracle's refined
reference solution: FP64 QR solve and the FP32-factor + FP64-refinement
mixed solve, on conditioned problems with large residuals.

Bounds. A backward-stable LS solve returns the exact solution of a problem
with ||dA|| <= eps ||A||, ||db|| <= eps ||b||; the LS perturbation bound
(Wedin; Higham, Accuracy and Stability, Thm. 20.1) then gives
  ||x - x^|| / ||x|| <= kappa eps / (1 - kappa eps) (2 + (kappa + 1) eta),
  eta = ||r|| / (||A|| ||x||)   (tan(theta) / (||A|| ||x|| / ||Ax||)),
and for the normal-equation residual (the same backward perturbation)
  ||A^T r^|| / (||A|| ||r^||) <= eps (1 + ||A|| ||x^|| / ||r^||).
eta is measured from the reference solution. Householder QR's normwise
backward error is O(u) in practice (the worst-case constant grows with mn
but is never approached: the GPU factorizations here measure well below
n u); eps = 4 u is used, which keeps the forward-error bound below 1e-8 at
kappa = 1e6 (5e-9 at 16384 x 4096, where the FP64 solve measures 1.5e-10)
while leaving a margin of more than 10x over the measured errors. The normal-equation residual is evaluated in long double so that
the check's own rounding (of order u ||A|| ||x|| / ||r||) does not mask it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1102_5328_gb300 import inputs

U = 2.0 ** -53
EPS = 4 * U  # normwise backward error of the QR solve (see above)


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
    # FP64-level forward error: at most twice the plain FP64 solve's, per RHS
    assert np.all(emx <= 2 * e64), (emx, e64)
    # FP64 path: within the LS perturbation bound with eps = 4u
    bound = perturbation_bound(A, B, Xref, kappa)
    assert np.all(e64 <= bound), (e64, bound)
    assert kappa < 1e6 or np.all(bound < 1e-8), bound


def perturbation_bound(A, B, Xref, kappa, eps=EPS):
    """kappa eps / (1 - kappa eps) (2 + (kappa + 1) eta) per column, eta
    measured from the reference solution. ||A||_2 = 1: the inputs are built
    as U diag(sigma) V^T with sigma_max = 1."""
    normA = 1.0
    R = B - A @ Xref
    eta = np.linalg.norm(R, axis=0) / (normA * np.linalg.norm(Xref, axis=0))
    ke = kappa * eps
    return ke / (1 - ke) * (2 + (kappa + 1) * eta)


def _normal_eq_ld(A, B, X):
    """||A^T r|| / (||A|| ||r||) with r = b - A x and A^T r formed in long
    double from the fp64 values of A, b and x."""
    Al = A.astype(np.longdouble)
    R = B.astype(np.longdouble) - Al @ X.astype(np.longdouble)
    AtR = (Al.T @ R).astype(np.float64)
    Rn = R.astype(np.float64)
    return np.linalg.norm(AtR, axis=0) / np.linalg.norm(Rn, axis=0), Rn  # ||A||_2 = 1


def test_normal_equations_residual(q):
    """The mixed solution satisfies the normal equations to the backward
    error of a stable solve: ||A^T r|| / (||A|| ||r||) <= eps (1 + ||A|| ||x||
    / ||r||), eps = 4u, evaluated in long double; and the FP64 QR solve too."""
    kappa = 1e6
    A, B = inputs.ls_problem(2048, 512, 4, kappa=kappa, seed=5)
    X, info = q.qr_solve_ls(to_dev(A), to_dev(B), prec=q.QR_PREC_F32, nb=128, ib=32, max_iter=50)
    X64, _ = q.qr_solve_ls(to_dev(A), to_dev(B), prec=q.QR_PREC_F64, nb=128, ib=32)
    normA = 1.0  # sigma_max of U diag(sigma) V^T
    for Xs in (X.cpu().numpy(), X64.cpu().numpy()):
        ne, R = _normal_eq_ld(A, B, Xs)
        bound = EPS * (1 + normA * np.linalg.norm(Xs, axis=0) / np.linalg.norm(R, axis=0))
        assert np.all(ne <= bound), (ne, bound)


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


@pytest.mark.slow
def test_least_squares_full_size(q):
    """The mixed-precision least-squares workload at full size: A 16384 x 4096
    = U diag(sigma) V^T with sigma geometric from 1 to 1e-6, 8 right-hand
    sides N(0, 1). The FP32-factor solve refined in FP64 reaches the FP64
    solve's forward error (within 2x, per RHS) against the oracle's
    doubled-precision refined solution, and the FP64 solve is within the
    perturbation bound (eps = 4u, below 1e-8 here)."""
    m, n, k, kappa = 16384, 4096, 8, 1e6
    A, B = inputs.ls_problem(m, n, k, kappa=kappa, seed=5)
    Xref, _ = oracle.ls_refine(A, B, maxit=30)
    Ad, Bd = to_dev(A), to_dev(B)
    X64, info64 = q.qr_solve_ls(Ad, Bd, prec=q.QR_PREC_F64)
    Xmx, infomx = q.qr_solve_ls(Ad, Bd, prec=q.QR_PREC_F32, max_iter=50)
    assert info64[2] == 0 and infomx[2] == 0 and infomx[1] in (1, 2), (info64, infomx)
    e64 = fwd_err(X64.cpu().numpy(), Xref)
    emx = fwd_err(Xmx.cpu().numpy(), Xref)
    assert np.all(emx <= 2 * e64), (emx, e64)
    bound = perturbation_bound(A, B, Xref, kappa)
    assert np.all(bound < 1e-8) and np.all(e64 <= bound), (e64, bound)


@pytest.fixture
def refine_option(q):
    yield lambda v: q.qr_set_option(q.QR_OPT_LS_REFINE, v)
    q.qr_set_option(q.QR_OPT_LS_REFINE, 0)


@pytest.mark.parametrize("prec,kappa,refine", [(3, 1e6, 0), (3, 1e4, 0), (2, 1e3, 0), (1, 1e6, 2)])
def test_gmres_ir_reaches_fp64_forward_error(q, refine_option, prec, kappa, refine):
    """GMRES-based refinement (FP64 GMRES on the augmented system,
    preconditioned by the low-precision QR): with BF16x3 tensor-core factors
    (u about 2^-17, kappa u up to 15 here), TF32 factors at kappa = 1e3 and,
    forced by QR_OPT_LS_REFINE = 2, FP32 factors, the solution reaches the
    FP64 solve's forward error (within 2x, per RHS). Large residuals (b ~
    N(0,1)), ragged sizes."""
    refine_option(refine)
    m, n = 1100, 450
    A, B = inputs.ls_problem(m, n, 3, kappa=kappa, seed=prec * 11 + int(np.log10(kappa)))
    Xref, _ = oracle.ls_refine(A, B, maxit=30)
    X64, _ = q.qr_solve_ls(to_dev(A), to_dev(B), prec=q.QR_PREC_F64, nb=64, ib=16)
    X, info = q.qr_solve_ls(to_dev(A), to_dev(B), prec=prec, nb=64, ib=16, max_iter=20, tol=1e-11)
    e64 = fwd_err(X64.cpu().numpy(), Xref)
    ex = fwd_err(X.cpu().numpy(), Xref)
    assert info[2] == 0 and info[1] in (1, 2) and info[3] > 0, info
    assert np.all(ex <= 2 * e64), (ex, e64, info)


def test_bf16x3_plain_refinement_does_not_converge_at_kappa_1e6(q, refine_option):
    """The reason GMRES-IR exists: with kappa u about 15 (BF16x3 factors,
    kappa = 1e6) Bjorck's augmented refinement, forced by QR_OPT_LS_REFINE
    = 1, stalls far from the FP64-level solution."""
    refine_option(1)
    m, n = 1100, 450
    A, B = inputs.ls_problem(m, n, 2, kappa=1e6, seed=77)
    Xref, _ = oracle.ls_refine(A, B, maxit=30)
    X, info = q.qr_solve_ls(to_dev(A), to_dev(B), prec=q.QR_PREC_BF16X3, nb=64, ib=16, max_iter=20, tol=1e-11)
    ex = fwd_err(X.cpu().numpy(), Xref)
    assert info[3] == 0 and np.all(ex > 1e-6), (ex, info)


@pytest.mark.slow
def test_least_squares_full_size_bf16x3_gmres(q):
    """The full-size least-squares workload with BF16x3 tensor-core factors
    and GMRES-IR: FP64-level forward error (within 2x of the FP64 solve)."""
    m, n, k, kappa = 16384, 4096, 8, 1e6
    A, B = inputs.ls_problem(m, n, k, kappa=kappa, seed=5)
    Xref, _ = oracle.ls_refine(A, B, maxit=30)
    Ad, Bd = to_dev(A), to_dev(B)
    X64, _ = q.qr_solve_ls(Ad, Bd, prec=q.QR_PREC_F64)
    X, info = q.qr_solve_ls(Ad, Bd, prec=q.QR_PREC_BF16X3, max_iter=20, tol=1e-11)
    e64 = fwd_err(X64.cpu().numpy(), Xref)
    ex = fwd_err(X.cpu().numpy(), Xref)
    assert info[2] == 0 and info[3] > 0, info
    assert np.all(ex <= 2 * e64), (ex, e64, info)
