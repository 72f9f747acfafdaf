"""Pins for the oracle's two accuracy checks, CPU only.

``oracle.fact_residual`` (||A - Q R||_F / ||A||_F) and ``oracle.orth_residual``
(||I - Q^T Q||_F) decide every GPU parity verdict against the acceptance
bounds (backward error and orthogonality <= 10 n u, the factorization problem
of Sec. 2.1). Each pin here fixes their value by something other than the
checkers themselves: exact rational arithmetic on small dyadic inputs (every
product and sum exact, so the long-double evaluation must agree to rounding of
the final square root), a Q that is exactly orthogonal, a known perturbation
Q (I + eps E) whose defect is known in closed form, and a single entry of R
changed by delta, whose residual is delta / ||A||_F.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


def _frac(M):
    return [[Fraction(float(x)) for x in row] for row in np.asarray(M).tolist()]


def _sqrt_frac(x):
    """sqrt of a non-negative Fraction to about 1e-17 relative."""
    if x == 0:
        return 0.0
    # one Newton step in Fractions from the double estimate
    y = Fraction(math.sqrt(float(x)))
    y = (y + x / y) / 2
    return float(y)


def _exact_fact_residual(A, Q, R):
    """||A - Q triu(R[:n, :n])||_F / ||A||_F in exact rationals (the entries
    of R below its diagonal do not belong to the factor and are ignored)."""
    Af, Qf, Rf = _frac(A), _frac(Q), _frac(R)
    m, n = len(Af), len(Af[0])
    num = Fraction(0)
    den = Fraction(0)
    for r in range(m):
        for c in range(n):
            s = Af[r][c] - sum(Qf[r][p] * Rf[p][c] for p in range(c + 1))
            num += s * s
            den += Af[r][c] * Af[r][c]
    return _sqrt_frac(num) / _sqrt_frac(den)


def _exact_orth_residual(Q):
    Qf = _frac(Q)
    m, n = len(Qf), len(Qf[0])
    acc = Fraction(0)
    for i in range(n):
        for j in range(n):
            s = (1 if i == j else 0) - sum(Qf[r][i] * Qf[r][j] for r in range(m))
            acc += s * s
    return _sqrt_frac(acc)


def _dyadic(rng, shape, lo=-8, hi=9, den=8):
    """Small dyadic rationals k / den: every product and sum of a few of them
    is exact in fp64 and long double."""
    return rng.integers(lo, hi, size=shape).astype(np.float64) / den


def _signed_permutation(rng, m):
    P = np.zeros((m, m))
    P[np.arange(m), rng.permutation(m)] = rng.choice([-1.0, 1.0], size=m)
    return P


@pytest.mark.parametrize("m,n,seed", [(5, 5, 0), (7, 4, 1), (9, 6, 2), (3, 1, 3)])
def test_fact_residual_exact_rational(m, n, seed):
    """Arbitrary (non-orthogonal) Q and R with dyadic entries; R carries
    garbage below its diagonal, which the check must ignore."""
    rng = np.random.default_rng(500 + seed)
    A = _dyadic(rng, (m, n))
    Q = _dyadic(rng, (m, n))
    R = _dyadic(rng, (n, n))
    want = _exact_fact_residual(A, Q, R)
    got = oracle.fact_residual(A, Q, R)
    assert want > 0.1
    assert abs(got - want) <= 1e-14 * want, (got, want)
    # the strictly lower triangle of R is not part of the factor
    R2 = R + np.tril(_dyadic(rng, (n, n)), -1)
    assert oracle.fact_residual(A, Q, R2) == got


@pytest.mark.parametrize("m,n,seed", [(6, 6, 0), (8, 5, 1), (4, 2, 2)])
def test_fact_residual_single_entry(m, n, seed):
    """A = P R0 with P a signed permutation (exactly orthogonal): the exact
    factors give 0, and R with one entry (i <= j) changed by delta gives
    delta / ||A||_F, since ||P e_i delta|| = delta."""
    rng = np.random.default_rng(600 + seed)
    P = _signed_permutation(rng, m)[:, :n]
    R0 = np.triu(_dyadic(rng, (n, n), 1, 9))
    A = P @ R0
    assert oracle.fact_residual(A, P, R0) == 0.0
    normA = math.sqrt(float(sum(Fraction(x) ** 2 for x in A.ravel().tolist())))
    for (i, j), delta in [((0, n - 1), 0.25), ((n - 1, n - 1), -1.5), ((n // 2, n // 2), 3.0)]:
        R = R0.copy()
        R[i, j] += delta
        got = oracle.fact_residual(A, P, R)
        assert abs(got - abs(delta) / normA) <= 1e-15 * abs(delta) / normA, (i, j, got)


@pytest.mark.parametrize("m,n,seed", [(4, 4, 0), (6, 3, 1), (8, 8, 2), (5, 1, 3)])
def test_orth_residual_exact_rational(m, n, seed):
    rng = np.random.default_rng(700 + seed)
    Q = _dyadic(rng, (m, n))
    want = _exact_orth_residual(Q)
    got = oracle.orth_residual(Q)
    assert abs(got - want) <= 1e-14 * want, (got, want)


@pytest.mark.parametrize("m,n,seed", [(6, 6, 0), (9, 5, 1)])
def test_orth_residual_perturbed(m, n, seed):
    """Q = P (I + eps E) with P a signed permutation: Q^T Q = (I + eps E)^T
    (I + eps E), so ||I - Q^T Q||_F = ||eps (E + E^T) + eps^2 E^T E||_F.
    With eps = 2^-20 and small integer E every entry is exact in fp64."""
    rng = np.random.default_rng(800 + seed)
    eps = 2.0 ** -20
    E = rng.integers(-3, 4, size=(n, n)).astype(np.float64)
    P = _signed_permutation(rng, m)[:, :n]
    Q = P @ (np.eye(n) + eps * E)
    assert np.array_equal(P.T @ Q, np.eye(n) + eps * E)  # the construction is exact
    Ef = [[Fraction(int(x)) for x in row] for row in E.tolist()]
    e = Fraction(1, 2 ** 20)
    acc = Fraction(0)
    for i in range(n):
        for j in range(n):
            d = e * (Ef[i][j] + Ef[j][i]) + e * e * sum(Ef[k][i] * Ef[k][j] for k in range(n))
            acc += d * d
    want = _sqrt_frac(acc)
    got = oracle.orth_residual(Q)
    assert abs(got - want) <= 1e-13 * want, (got, want)
    # an exactly orthogonal Q has no defect at all
    assert oracle.orth_residual(P) == 0.0


def test_orth_residual_scaled_columns():
    """Columns of norm (1 + a_j), mutually orthogonal: the defect is
    sqrt(sum_j (2 a_j + a_j^2)^2), a pure-diagonal case."""
    a = np.array([0.5, -0.25, 0.125, 0.0])
    Q = np.vstack([np.diag(1.0 + a), np.zeros((2, 4))])
    want = math.sqrt(float(sum(Fraction(2 * x + x * x) ** 2 for x in a.tolist())))
    assert abs(oracle.orth_residual(Q) - want) <= 1e-15 * want
