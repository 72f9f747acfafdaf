"""CPU oracle for the tile Householder QR path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package. The GPU
product path (``paper_1102_5328_gb300``) never imports it, and this package
imports nothing from the product path.

Contents:
  * ``qr_oracle.c`` -- unblocked fp64 Householder QR (dgeqr2-style), explicit
    Q, Q^T/Q application, back substitution, QR least squares, a
    doubled-precision augmented-system refinement (reference LS solution),
    long-double modified Gram-Schmidt (brute-force pin) and long-double
    accuracy checks; the column-by-column Cholesky A = L L^T and its
    long-double residual. Built with gcc into ``oracle/_build/liboracle.so``.
  * ``tuning.py`` -- the paper's pruning rules (Properties 5.1, 4.2, 5.1,
    Heuristics 0/1/2, nearest-point interpolation) as plain Python loops.
  * ``mlp.py`` -- fp64 numpy forward/backward/Adam of the cost-model MLP.
  * ``tile_apply.py`` -- Q^T of a flat-tree tile QR applied in NumPy from
    stored factors (reflectors and T blocks): the large-N probe that checks
    the GPU's stored factors independently of its Q-application kernels.
  * ``lu.py`` -- tile LU with incremental (pairwise) pivoting written out task
    by task (GETRF, GESSM, TSTRF, SSSSM) with NumPy row operations, the
    transformations applied to other columns, back substitution.

The paper is Agullo, Dongarra, Nath, Tomov, "A Fully Empirical Autotuned
Dense QR Factorization for Multicore Architectures" (INRIA RR-7526).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "qr_oracle.c")

_lib = None


def build(force=False):
    """Compile the C oracle with gcc (OpenMP, no fp contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        i64, dp, i32 = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        L.oracle_set_threads.argtypes = [i32]
        L.oracle_geqr2.argtypes = [i64, i64, i64, dp, i64, dp]
        L.oracle_apply_qt.argtypes = [i64, i64, dp, i64, dp, i64, dp, i64]
        L.oracle_apply_q.argtypes = [i64, i64, dp, i64, dp, i64, dp, i64]
        L.oracle_form_q.argtypes = [i64, i64, dp, i64, dp, dp, i64]
        L.oracle_trsm_upper.argtypes = [i64, dp, i64, i64, dp, i64]
        L.oracle_ls_solve.argtypes = [i64, i64, dp, i64, i64, dp, i64, dp, i64]
        L.oracle_ls_refine.argtypes = [i64, i64, dp, i64, i64, dp, i64, dp, i64, i32, ctypes.c_double]
        L.oracle_mgs_ld.argtypes = [i64, i64, dp, i64, dp, i64]
        L.oracle_fact_residual.argtypes = [i64, i64, dp, i64, dp, i64, dp, i64]
        L.oracle_fact_residual.restype = ctypes.c_double
        L.oracle_orth_residual.argtypes = [i64, i64, dp, i64]
        L.oracle_orth_residual.restype = ctypes.c_double
        L.oracle_potrf.argtypes = [i64, dp, i64]
        L.oracle_chol_residual.argtypes = [i64, dp, i64, dp, i64]
        L.oracle_chol_residual.restype = ctypes.c_double
        _lib = L
    return _lib


def _f64(a):
    """Column-major (Fortran-ordered) fp64 copy."""
    return np.array(a, dtype=np.float64, order="F", copy=True)


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n):
    """Set the OpenMP thread count; returns the count in effect."""
    return lib().oracle_set_threads(int(n))


def geqr2(A, kmax=None):
    """Householder QR of A (m x n, m >= n or not). Returns (F, tau): R in the
    upper triangle of F, reflectors below it (LAPACK dgeqr2 storage).
    ``kmax`` limits the number of reflectors (partial factorization)."""
    F = _f64(A)
    m, n = F.shape
    k = min(m, n) if kmax is None else int(kmax)
    tau = np.zeros(max(k, 1))
    rc = lib().oracle_geqr2(m, n, k, _p(F), max(m, 1), _p(tau))
    assert rc == 0, rc
    return F, tau[:k]


def r_factor(F, k=None):
    """Upper-triangular R (k x n) from geqr2 storage."""
    m, n = F.shape
    k = min(m, n) if k is None else k
    return np.triu(F[:k, :])


def form_q(F, tau):
    """Explicit thin Q (m x n) from geqr2 storage."""
    m, n = F.shape
    k = len(tau)
    Q = np.zeros((m, k), order="F")
    Fc = _f64(F)
    t = np.ascontiguousarray(tau, dtype=np.float64)
    lib().oracle_form_q(m, k, _p(Fc), m, _p(t), _p(Q), m)
    return Q


def apply_qt(F, tau, C):
    """Q^T C for Q from geqr2 storage."""
    Fc = _f64(F)
    Cc = _f64(C.reshape(C.shape[0], -1))
    t = np.ascontiguousarray(tau, dtype=np.float64)
    lib().oracle_apply_qt(Fc.shape[0], len(t), _p(Fc), Fc.shape[0], _p(t), Cc.shape[1], _p(Cc), Cc.shape[0])
    return Cc.reshape(C.shape)


def apply_q(F, tau, C):
    """Q C for Q from geqr2 storage."""
    Fc = _f64(F)
    Cc = _f64(C.reshape(C.shape[0], -1))
    t = np.ascontiguousarray(tau, dtype=np.float64)
    lib().oracle_apply_q(Fc.shape[0], len(t), _p(Fc), Fc.shape[0], _p(t), Cc.shape[1], _p(Cc), Cc.shape[0])
    return Cc.reshape(C.shape)


def trsm_upper(R, Y):
    """Solve R X = Y for upper-triangular R (n x n)."""
    Rc = _f64(R)
    Yc = _f64(Y.reshape(Y.shape[0], -1))
    n = Rc.shape[1]
    lib().oracle_trsm_upper(n, _p(Rc), Rc.shape[0], Yc.shape[1], _p(Yc), Yc.shape[0])
    return Yc.reshape(Y.shape)


def ls_solve(A, B):
    """min ||A X - B|| by Householder QR (no refinement)."""
    Ac = _f64(A)
    Bc = _f64(B.reshape(B.shape[0], -1))
    m, n = Ac.shape
    X = np.zeros((n, Bc.shape[1]), order="F")
    rc = lib().oracle_ls_solve(m, n, _p(Ac), m, Bc.shape[1], _p(Bc), m, _p(X), n)
    assert rc == 0, rc
    return X.reshape((n,) + B.shape[1:])


def ls_refine(A, B, maxit=10, tol=2.0 ** -60):
    """Reference LS solution: QR solve refined on the augmented system with
    doubled-precision residuals. Returns (X, iterations)."""
    Ac = _f64(A)
    Bc = _f64(B.reshape(B.shape[0], -1))
    m, n = Ac.shape
    X = np.zeros((n, Bc.shape[1]), order="F")
    it = lib().oracle_ls_refine(m, n, _p(Ac), m, Bc.shape[1], _p(Bc), m, _p(X), n, int(maxit), float(tol))
    assert it >= 0, it
    return X.reshape((n,) + B.shape[1:]), it


def mgs_ld(A):
    """R of a long-double modified Gram-Schmidt (positive diagonal)."""
    Ac = _f64(A)
    m, n = Ac.shape
    R = np.zeros((n, n), order="F")
    lib().oracle_mgs_ld(m, n, _p(Ac), m, _p(R), n)
    return R


def fact_residual(A, Q, R):
    """||A - Q R||_F / ||A||_F in long double."""
    Ac, Qc, Rc = _f64(A), _f64(Q), _f64(R)
    m, n = Ac.shape
    return lib().oracle_fact_residual(m, n, _p(Ac), m, _p(Qc), Qc.shape[0], _p(Rc), Rc.shape[0])


def orth_residual(Q):
    """||I - Q^T Q||_F in long double."""
    Qc = _f64(Q)
    m, n = Qc.shape
    return lib().oracle_orth_residual(m, n, _p(Qc), m)


def potrf(A):
    """Cholesky A = L L^T by the column definition. Returns (L, info): L the
    lower triangle (zero above), info 0 or the 1-based column whose pivot was
    not positive."""
    F = _f64(A)
    n = F.shape[0]
    info = lib().oracle_potrf(n, _p(F), max(n, 1))
    return np.tril(F), info


def chol_residual(A, L):
    """||A - L L^T||_F / ||A||_F in long double (L: its lower triangle)."""
    Ac, Lc = _f64(A), _f64(L)
    n = Ac.shape[0]
    return lib().oracle_chol_residual(n, _p(Ac), n, _p(Lc), n)


def chol_flops(n):
    """Credited flops of a Cholesky factorization, n^3 / 3."""
    return float(n) ** 3 / 3.0


def qr_flops(m, n):
    """The credited flop count 2mn^2 - 2n^3/3 (= 4/3 N^3 for m = n, the
    performance definition of Sec. 2.2, independent of IB)."""
    m, n = float(m), float(n)
    return 2.0 * m * n * n - 2.0 * n ** 3 / 3.0


def row_signs(R_test, R_ref):
    """D = diag(sign(r_ii^test * r_ii^ref)) (+1 where either is zero)."""
    d = np.sign(np.diag(R_test) * np.diag(R_ref))
    d[d == 0] = 1.0
    return d
