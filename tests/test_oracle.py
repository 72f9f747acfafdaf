"""Pins for the CPU oracle (oracle/qr_oracle.c), CPU only.

Each test ties the oracle to something other than itself: a hand-derived
closed form, a matrix built from known factors, exact rational arithmetic,
invariants of the QR factorization, or a long-double Gram-Schmidt run.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1102_5328_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -53


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = [float(v) for v in vals]
    return out


def test_closed_form_2x2():
    g = _golden("householder_2x2.txt")
    A = np.array(g["A"]).reshape(2, 2)
    F, tau = oracle.geqr2(A)
    R = np.triu(F)
    # beta, tau and v are exact in fp64 (correctly rounded divisions of
    # integers); -2.2 and 0.4 come from 1 - 3.2 and 2 - 1.6, a few ulps off.
    assert R[0, 0] == -5.0 and R[1, 0] == 0.0
    assert np.allclose(R, np.array(g["R"]).reshape(2, 2), rtol=4 * U, atol=0)
    assert np.array_equal(tau, np.array(g["tau"]))
    assert F[1, 0] == g["v1"][0]
    Q = oracle.form_q(F, tau)
    assert np.isclose(np.linalg.det(Q), -1.0, atol=1e-15)
    assert np.allclose(Q @ R, A, atol=4 * U)


def _rational_reflector(v):
    """H = I - 2 v v^T / (v^T v): orthogonal and exactly rational for integer v."""
    v = [Fraction(int(x)) for x in v]
    vv = sum(x * x for x in v)
    n = len(v)
    return [[(1 if i == j else 0) - 2 * v[i] * v[j] / vv for j in range(n)] for i in range(n)]


def _matmul_frac(A, B):
    return [[sum(A[i][k] * B[k][j] for k in range(len(B))) for j in range(len(B[0]))] for i in range(len(A))]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_constructed_q0_r0(seed):
    """A = Q0 R0 with Q0 a product of exactly-rational reflectors and R0 upper
    triangular: Householder QR must return R0 up to row signs."""
    rng = np.random.default_rng(100 + seed)
    m, n = 9, 6
    Q0 = [[Fraction(1 if i == j else 0) for j in range(m)] for i in range(m)]
    for _ in range(3):
        Q0 = _matmul_frac(Q0, _rational_reflector(rng.integers(-4, 5, size=m) + np.eye(m)[rng.integers(m)]))
    R0 = [[Fraction(0)] * n for _ in range(m)]
    for i in range(n):
        R0[i][i] = Fraction(int(rng.integers(1, 6)))
        for j in range(i + 1, n):
            R0[i][j] = Fraction(int(rng.integers(-5, 6)), 2)
    A = np.array([[float(x) for x in row] for row in _matmul_frac(Q0, R0)])
    R0f = np.array([[float(x) for x in row] for row in R0])[:n]
    F, tau = oracle.geqr2(A)
    R = np.triu(F[:n])
    D = np.sign(np.diag(R)) * np.sign(np.diag(R0f))
    assert np.all(D != 0)
    err = np.abs(D[:, None] * R - R0f).max() / np.abs(R0f).max()
    assert err < 64 * U, err
    # Q's first n columns are Q0's up to the same signs
    Q = oracle.form_q(F, tau)
    Q0f = np.array([[float(x) for x in row] for row in Q0])[:, :n]
    assert np.abs(Q * D[None, :] - Q0f).max() < 64 * U


def test_trivial_cases():
    # diagonal: every reflector is the identity, R = A exactly
    A = np.diag([3.0, -2.0, 0.5, 7.0])
    F, tau = oracle.geqr2(A)
    assert np.all(tau == 0.0) and np.array_equal(F, A)
    # upper triangular, tall: the zero rows below keep every tau = 0
    rng = np.random.default_rng(3)
    A = np.vstack([np.triu(rng.standard_normal((5, 5))), np.zeros((3, 5))])
    F, tau = oracle.geqr2(A)
    assert np.all(tau == 0.0) and np.array_equal(F, A)
    # a zero column: tau = 0 there and that column of R stays zero
    A = rng.standard_normal((6, 4))
    A[:, 0] = 0.0
    F, tau = oracle.geqr2(A)
    assert tau[0] == 0.0 and np.all(F[:, 0] == 0.0)


def test_rtr_equals_ata():
    A = inputs.uniform_matrix(40, 25, seed=7)
    F, tau = oracle.geqr2(A)
    R = np.triu(F[:25])
    # exact A^T A in rationals (fp64 values are exact rationals)
    Af = [[Fraction(x) for x in row] for row in A.T.tolist()]
    AtA = np.array([[float(sum(a * b for a, b in zip(Af[i], Af[j]))) for j in range(25)] for i in range(25)])
    err = np.abs(R.T @ R - AtA).max() / np.abs(AtA).max()
    assert err < 25 * 10 * U, err


@pytest.mark.parametrize("m,n", [(8, 8), (8, 5), (6, 3), (3, 3), (1, 1), (5, 1)])
def test_against_long_double_mgs(m, n):
    rng = np.random.default_rng(m * 10 + n)
    A = rng.random((m, n)) - 0.5
    F, tau = oracle.geqr2(A)
    R = np.triu(F[:n])
    Rm = oracle.mgs_ld(A)
    R_pos = R * np.sign(np.diag(R))[:, None]
    assert np.abs(R_pos - Rm).max() < 100 * U * max(1.0, np.abs(Rm).max())


@pytest.mark.parametrize("m,n", [(128, 128), (300, 200), (513, 130)])
def test_backward_and_orthogonality(m, n):
    A = inputs.uniform_matrix(m, n, seed=m + n)
    F, tau = oracle.geqr2(A)
    Q = oracle.form_q(F, tau)
    R = np.triu(F[:n])
    assert oracle.fact_residual(A, Q, R) / (n * U) <= 10.0
    assert oracle.orth_residual(Q) / (n * U) <= 10.0
    # Q^T A = R through the applier
    QtA = oracle.apply_qt(F, tau, A.copy())
    assert np.abs(QtA[:n] - R).max() < 50 * n * U
    if m > n:
        assert np.abs(QtA[n:]).max() < 50 * n * U
    # Q (Q^T C) = C
    C = inputs.normal_matrix(m, 3, seed=1)
    assert np.abs(oracle.apply_q(F, tau, oracle.apply_qt(F, tau, C)) - C).max() < 50 * n * U


def test_partial_factorization_rows_final():
    A = inputs.uniform_matrix(200, 150, seed=11)
    F_full, _ = oracle.geqr2(A)
    F_part, tau = oracle.geqr2(A, kmax=20)
    assert len(tau) == 20
    assert np.array_equal(np.triu(F_part[:20]), np.triu(F_full[:20]))


def _exact_ls(A, b):
    """Exact least-squares solution of the rational normal equations."""
    Af = [[Fraction(x) for x in row] for row in A.tolist()]
    bf = [Fraction(x) for x in b.tolist()]
    m, n = len(Af), len(Af[0])
    M = [[sum(Af[k][i] * Af[k][j] for k in range(m)) for j in range(n)] for i in range(n)]
    r = [sum(Af[k][i] * bf[k] for k in range(m)) for i in range(n)]
    for c in range(n):  # Gauss-Jordan, exact
        p = next(i for i in range(c, n) if M[i][c] != 0)
        M[c], M[p], r[c], r[p] = M[p], M[c], r[p], r[c]
        for i in range(n):
            if i != c and M[i][c] != 0:
                f = M[i][c] / M[c][c]
                M[i] = [a - f * b_ for a, b_ in zip(M[i], M[c])]
                r[i] -= f * r[c]
    return np.array([float(r[i] / M[i][i]) for i in range(n)])


def test_ls_solve_and_refinement_exact():
    """A kappa = 1e5 problem with a large residual: the refined solution must
    equal the exact rational LS solution to a few ulps; the plain QR solve is
    allowed the kappa^2 * u * tan(theta) error of fp64 LS."""
    A, B = inputs.ls_problem(12, 5, 2, kappa=1e5, seed=21)
    X, it = oracle.ls_refine(A, B, maxit=20)
    X0 = oracle.ls_solve(A, B)
    for c in range(2):
        xs = _exact_ls(A, B[:, c])
        rel = np.linalg.norm(X[:, c] - xs) / np.linalg.norm(xs)
        assert rel < 8 * U, rel
        rel0 = np.linalg.norm(X0[:, c] - xs) / np.linalg.norm(xs)
        assert rel0 < 1e5 ** 2 * 100 * U
    assert 1 <= it <= 20


def test_ls_consistent_system():
    A = inputs.uniform_matrix(60, 20, seed=5)
    x0 = inputs.normal_matrix(20, 1, seed=6)[:, 0]
    b = A @ x0
    x = oracle.ls_solve(A, b[:, None])[:, 0]
    assert np.linalg.norm(x - x0) / np.linalg.norm(x0) < 1e3 * U * np.linalg.cond(A)


def test_flop_credit():
    g = _golden("performance_metric.txt")
    N = g["N"][0]
    assert oracle.qr_flops(N, N) == pytest.approx(4.0 / 3.0 * N ** 3, rel=1e-15)
    # 272.55 / 537.6 = 50.7 % quoted for the Istanbul optimum at N = 6000
    assert round(100 * g["gflops"][0] / g["peak"][0], 1) == 50.7
