"""Pins for the oracle's Cholesky factorization (oracle_potrf) and its
residual check (oracle_chol_residual), CPU only: a hand-derived 3x3 closed
form, exact recovery of A = L0 L0^T for integer L0 with power-of-two
diagonals (every step exact), agreement with LAPACK's Cholesky (NumPy) on
well-conditioned matrices, the residual check on exact rational cases, and
the detection of matrices that are not positive definite."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -53


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, *v = line.split()
                out[k] = [float(x) for x in v]
    return out


def test_closed_form_3x3():
    g = _golden("cholesky_3x3.txt")
    A = np.array(g["A"]).reshape(3, 3)
    L, info = oracle.potrf(A)
    assert info == 0
    assert np.array_equal(L, np.array(g["L"]).reshape(3, 3))


def _integer_factor(rng, n):
    L0 = np.tril(rng.integers(-3, 4, size=(n, n)).astype(np.float64), -1)
    L0 += np.diag(rng.choice([1.0, 2.0, 4.0], size=n))
    return L0


@pytest.mark.parametrize("n,seed", [(5, 0), (9, 1), (16, 2)])
def test_exact_recovery(n, seed):
    """A = L0 L0^T with small integers and diagonals in {1, 2, 4}: sums of
    integer products, square roots of perfect squares and divisions by powers
    of two are all exact, so the oracle returns L0 exactly."""
    L0 = _integer_factor(np.random.default_rng(900 + seed), n)
    A = L0 @ L0.T
    L, info = oracle.potrf(A)
    assert info == 0 and np.array_equal(L, L0)
    assert oracle.chol_residual(A, L) == 0.0


@pytest.mark.parametrize("n", [1, 40, 130])
def test_against_lapack(n):
    rng = np.random.default_rng(n)
    G = rng.standard_normal((n, n))
    A = G @ G.T / n + np.eye(n)
    L, info = oracle.potrf(A)
    Lr = np.linalg.cholesky(A)
    assert info == 0
    assert np.linalg.norm(L - Lr) / np.linalg.norm(Lr) <= 20 * n * U
    assert oracle.chol_residual(A, L) <= 10 * n * U


def test_residual_exact_rational():
    """||A - L L^T||_F / ||A||_F against exact rationals: an arbitrary dyadic
    L (not a factor of A), whose upper triangle must be ignored."""
    rng = np.random.default_rng(11)
    n = 6
    A = rng.integers(-8, 9, size=(n, n)).astype(np.float64) / 4
    A = A + A.T
    L = np.tril(rng.integers(-8, 9, size=(n, n)).astype(np.float64) / 8)
    Lg = L + np.triu(rng.integers(-8, 9, size=(n, n)).astype(np.float64), 1)
    Af = [[Fraction(x) for x in row] for row in A.tolist()]
    Lf = [[Fraction(x) for x in row] for row in L.tolist()]
    num = den = Fraction(0)
    for i in range(n):
        for j in range(n):
            s = Af[i][j] - sum(Lf[i][k] * Lf[j][k] for k in range(n))
            num += s * s
            den += Af[i][j] ** 2
    want = math.sqrt(float(num)) / math.sqrt(float(den))
    got = oracle.chol_residual(A, Lg)
    assert abs(got - want) <= 1e-14 * want


def test_single_entry_perturbation():
    """Changing L_ij (i > j) of an exact factor by delta changes L L^T in
    row/column i by delta * L[:, j]: the residual is the norm of that
    symmetric rank-2 correction plus delta^2 on the diagonal, computed here
    exactly."""
    L0 = _integer_factor(np.random.default_rng(12), 7)
    A = L0 @ L0.T
    L = L0.copy()
    i, j, d = 5, 2, 0.5
    L[i, j] += d
    E = L @ L.T - A  # exact: small dyadics
    want = np.sqrt(np.sum(E * E)) / np.sqrt(np.sum(A * A))
    assert abs(oracle.chol_residual(A, L) - want) <= 1e-15 * want


def test_not_positive_definite():
    L0 = _integer_factor(np.random.default_rng(13), 6)
    A = L0 @ L0.T
    A[3, 3] -= 1000.0  # the pivot of column 3 becomes negative
    _, info = oracle.potrf(A)
    assert info == 4
    _, info = oracle.potrf(np.zeros((3, 3)))
    assert info == 1
