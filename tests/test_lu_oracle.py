"""Pins for the oracle's tile LU with incremental pivoting (CPU only).

* A hand-derived 3x3 (tests/golden/lu_incpiv_3x3.txt) with tiles of order 1
  (pairwise pivoting at every step) and of order 3 (partial pivoting): exact
  factors, pivot records and solution.
* The factorization's own transformations take A to the upper triangle of
  its result (the defining property of the factors) at ragged tile sizes.
* One tile is LU with partial pivoting: U equals LAPACK's (scipy) U.
* Solutions agree with LAPACK's solve within the conditioning bound; a zero
  column is reported by info; planted mistakes fail the pins.
* A column diagonally dominant matrix needs no swap anywhere, and the tile
  factors equal the textbook unpivoted right-looking LU bit for bit.
"""
import os
import types

import numpy as np
import pytest

from oracle import lu

HERE = os.path.dirname(os.path.abspath(__file__))
U = 2.0 ** -53


def _golden():
    vals, pivs = {}, {}
    with open(os.path.join(HERE, "golden", "lu_incpiv_3x3.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *rest = line.split()
            if key.startswith("piv_"):
                pivs[key] = {tuple(int(v) for v in t.split("=")[0].strip("()").split(",")): int(t.split("=")[1])
                             for t in rest}
            else:
                vals[key] = np.array([float(v) for v in rest])
    return vals, pivs


def test_golden_3x3_pairwise_and_partial():
    vals, pivs = _golden()
    A = vals["A"].reshape(3, 3)
    for nb, key in ((1, "piv_nb1"), (3, "piv_nb3")):
        F, piv, info = lu.getrf_incpiv(A, nb)
        assert info == 0
        assert np.array_equal(F, vals["F"].reshape(3, 3)), (nb, F)
        for (i, k, c), v in pivs[key].items():
            assert piv[i, k, c] == v, (nb, i, k, c)
        assert np.array_equal(lu.lu_solve(F, piv, nb, vals["b"])[:, 0], vals["x"])
    assert np.prod(np.diag(vals["F"].reshape(3, 3))) == -21.5


def _random(n, seed):
    return np.random.default_rng(seed).uniform(-0.5, 0.5, (n, n))


@pytest.mark.parametrize("n,nb", [(50, 7), (64, 16), (33, 40), (96, 32), (5, 1), (70, 64)])
def test_transformations_take_a_to_u(n, nb):
    A = _random(n, n + nb)
    F, piv, info = lu.getrf_incpiv(A, nb)
    assert info == 0
    Y = lu.apply_incpiv(F, piv, nb, A)
    nA = np.abs(A).max()
    assert np.abs(np.triu(Y) - np.triu(F)).max() <= 50 * n * U * nA
    assert np.abs(np.tril(Y, -1)).max() <= 50 * n * U * nA
    # every TSTRF pivot record is a row of the tile below or -1; GETRF's a row of the tile
    NT = (n + nb - 1) // nb
    for k in range(NT):
        nk = min(nb, n - k * nb)
        assert all(c <= piv[k, k, c] < nk for c in range(nk))
        for i in range(k + 1, NT):
            ni = min(nb, n - i * nb)
            assert all(-1 <= piv[i, k, c] < ni for c in range(nk))


def test_one_tile_is_partial_pivoting():
    sl = pytest.importorskip("scipy.linalg")
    A = _random(40, 3)
    F, piv, _ = lu.getrf_incpiv(A, 64)
    P, L, Ul = sl.lu(A)
    assert np.abs(np.triu(F) - Ul).max() <= 1e-13
    # the row chosen at each column is LAPACK's: P^T A's row order
    order = list(range(40))
    for c in range(40):
        p = piv[0, 0, c]
        order[c], order[p] = order[p], order[c]
    assert np.array_equal(np.argmax(P, axis=0), np.array(order))


@pytest.mark.parametrize("n,nb", [(64, 16), (100, 24), (128, 32)])
def test_solve_matches_lapack(n, nb):
    A = _random(n, 7 * n)
    b = np.random.default_rng(n).standard_normal((n, 2))
    F, piv, _ = lu.getrf_incpiv(A, nb)
    x = lu.lu_solve(F, piv, nb, b)
    ref = np.linalg.solve(A, b)
    kappa = np.linalg.cond(A)
    assert np.abs(x - ref).max() / np.abs(ref).max() <= 100 * n * kappa * U
    assert np.abs(A @ x - b).max() <= 100 * n * U * np.abs(A).max() * np.abs(x).max()


def test_zero_column_reported():
    A = _random(20, 5)
    A[:, 13] = 0.0
    _, _, info = lu.getrf_incpiv(A, 8)
    assert info == 14


MUTANTS = [
    # TSTRF takes the bottom row on ties too
    ("if abs(B[r, c]) > abs(T[c, c]):", "if abs(B[r, c]) >= abs(T[c, c]):"),
    # SSSSM forgets its row swap
    ("                    if r >= 0:\n                        tmp = X[c, :].copy()\n                        X[c, :] = Y[r, :]\n"
     "                        Y[r, :] = tmp\n                    Y -= np.outer(B[:, c], X[c, :])\n    return F, piv, info",
     "                    Y -= np.outer(B[:, c], X[c, :])\n    return F, piv, info"),
    # GETRF swaps the whole rows (multipliers included)
    ("                T[[c, p], c:] = T[[p, c], c:]\n            d = T[c, c]",
     "                T[[c, p], :] = T[[p, c], :]\n            d = T[c, c]"),
    # the trailing update adds instead of subtracting
    ("            B[:, c + 1:] -= np.outer(B[:, c], T[c, c + 1:])", "            B[:, c + 1:] += np.outer(B[:, c], T[c, c + 1:])"),
]


@pytest.mark.parametrize("old,new", MUTANTS)
def test_mutants_fail_a_pin(old, new):
    src = open(lu.__file__).read()
    assert src.count(old) == 1, old
    mod = types.ModuleType("lu_mutant")
    exec(compile(src.replace(old, new), "lu_mutant", "exec"), mod.__dict__)
    failed = False
    vals, pivs = _golden()
    A3 = vals["A"].reshape(3, 3)
    for nb in (1, 3):
        F, piv, _ = mod.getrf_incpiv(A3, nb)
        failed |= not np.array_equal(F, vals["F"].reshape(3, 3))
    A = _random(50, 57)
    A[3, 0] = A[40, 0] = 2.0  # a tie between the diagonal tile and a tile below in column 0
    A[0, 0] = 2.0
    F, piv, _ = mod.getrf_incpiv(A, 7)
    Y = mod.apply_incpiv(F, piv, 7, A)
    failed |= np.abs(np.tril(Y, -1)).max() > 1e-10
    F0, _, _ = lu.getrf_incpiv(A, 7)
    failed |= not np.allclose(F, F0)
    assert failed


@pytest.mark.parametrize("n,nb", [(30, 7), (64, 16), (50, 50)])
def test_diagonally_dominant_is_unpivoted_lu(n, nb):
    """A strictly column diagonally dominant matrix keeps that property in
    every Schur complement, so no step swaps (GETRF keeps row c, TSTRF keeps
    U's row) and each entry sees the same subtractions in the same order as
    in the textbook right-looking LU without pivoting: the factors agree
    bit for bit."""
    rng = np.random.default_rng(n + nb)
    A = rng.uniform(-1.0, 1.0, (n, n))
    A[np.arange(n), np.arange(n)] = np.abs(A).sum(axis=0) + 1.0
    F, piv, info = lu.getrf_incpiv(A, nb)
    assert info == 0
    NT = (n + nb - 1) // nb
    for k in range(NT):
        nk = min(nb, n - k * nb)
        assert all(piv[k, k, c] == c for c in range(nk))
        assert all((piv[i, k, :nk] == -1).all() for i in range(k + 1, NT))
    D = A.copy()
    for c in range(n):
        D[c + 1:, c] = D[c + 1:, c] / D[c, c]
        for r in range(c + 1, n):
            for j in range(c + 1, n):
                D[r, j] = D[r, j] - D[r, c] * D[c, j]
    assert np.array_equal(F, D)
