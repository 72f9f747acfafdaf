"""Tile LU with incremental (pairwise) pivoting -- TEST INFRASTRUCTURE ONLY.

The paper names LU next to Cholesky as a factorization its tile framework
and its tuning method carry over to (Secs. 1 and 7) and defines neither.
This is the tile LU of the same flat-tree DAG as the tile QR, with pivoting
restricted to what each tile task sees, written out task by task in program
order with plain NumPy row operations:

  GETRF(k)     A_kk = L_kk U_kk: column c takes the largest |entry| of
               rows c.. of the tile as pivot (first one on ties), swaps it
               with row c over columns c.., divides the column below by the
               pivot and subtracts the rank-1 product from the trailing block.
  GESSM(k, j)  the same row swaps and eliminations applied to A_kj.
  TSTRF(i, k)  the pair [U_kk; A_ik]: column c takes the largest |entry| of
               column c of A_ik when it exceeds |U_kk(c, c)| strictly (first
               one on ties), swaps that row with row c of U_kk over columns
               c.., divides A_ik's column c by the pivot and subtracts the
               rank-1 product from A_ik's columns c+1...
  SSSSM(i,j,k) the same swaps (row c of A_kj with the chosen row of A_ij)
               and eliminations applied to the pair [A_kj; A_ij].

Only the columns c.. take part in a swap, so each stored multiplier column
is the one its elimination step used; the factors are the sequence of these
elementary transformations (not L of one permutation of A) and the upper
triangle of the result is U. piv[i, k, c]: GETRF (i = k) the tile row
swapped with c (c itself when none); TSTRF (i > k) the row of A_ik swapped
with row c of U_kk, -1 when none.
"""
import numpy as np


def _blocks(n, nb):
    return [slice(s, min(n, s + nb)) for s in range(0, n, nb)]


def getrf_incpiv(A, nb):
    """(F, piv, info): F holds U on and above the diagonal and the
    multipliers below it; info = 1 + the first column whose pivot is 0
    (0 when none), as LAPACK's getrf reports it."""
    F = np.array(A, dtype=np.float64, copy=True)
    n = F.shape[0]
    assert F.shape == (n, n) and nb >= 1
    blk = _blocks(n, nb)
    NT = len(blk)
    piv = np.full((NT, NT, nb), -1, dtype=np.int64)
    info = 0
    for k in range(NT):
        K = blk[k]
        nk = K.stop - K.start
        T = F[K, K]  # a view
        # GETRF(k)
        for c in range(nk):
            p = c + int(np.argmax(np.abs(T[c:, c])))
            piv[k, k, c] = p
            if p != c:
                T[[c, p], c:] = T[[p, c], c:]
            d = T[c, c]
            if d == 0.0:
                info = info or K.start + c + 1
                continue
            T[c + 1:, c] /= d
            T[c + 1:, c + 1:] -= np.outer(T[c + 1:, c], T[c, c + 1:])
        # GESSM(k, j)
        for j in range(k + 1, NT):
            X = F[K, blk[j]]
            for c in range(nk):
                p = piv[k, k, c]
                if p != c:
                    X[[c, p], :] = X[[p, c], :]
                X[c + 1:, :] -= np.outer(T[c + 1:, c], X[c, :])
        for i in range(k + 1, NT):
            B = F[blk[i], K]
            # TSTRF(i, k)
            for c in range(nk):
                r = int(np.argmax(np.abs(B[:, c])))
                if abs(B[r, c]) > abs(T[c, c]):
                    piv[i, k, c] = r
                    tmp = T[c, c:].copy()
                    T[c, c:] = B[r, c:]
                    B[r, c:] = tmp
                d = T[c, c]
                if d == 0.0:
                    info = info or K.start + c + 1
                    continue
                B[:, c] /= d
                B[:, c + 1:] -= np.outer(B[:, c], T[c, c + 1:])
            # SSSSM(i, j, k)
            for j in range(k + 1, NT):
                X, Y = F[K, blk[j]], F[blk[i], blk[j]]
                for c in range(nk):
                    r = piv[i, k, c]
                    if r >= 0:
                        tmp = X[c, :].copy()
                        X[c, :] = Y[r, :]
                        Y[r, :] = tmp
                    Y -= np.outer(B[:, c], X[c, :])
    return F, piv, info


def apply_incpiv(F, piv, nb, C):
    """The factorization's transformations, in program order, applied to the
    rows of C (n x k): C -> L^-1 P C in the incremental-pivoting sense, so
    that A itself goes to U."""
    C = np.array(C, dtype=np.float64, copy=True)
    if C.ndim == 1:
        C = C[:, None]
    n = F.shape[0]
    blk = _blocks(n, nb)
    NT = len(blk)
    for k in range(NT):
        K = blk[k]
        nk = K.stop - K.start
        T, X = F[K, K], C[K]
        for c in range(nk):
            p = piv[k, k, c]
            if p != c:
                X[[c, p], :] = X[[p, c], :]
            X[c + 1:, :] -= np.outer(T[c + 1:, c], X[c, :])
        for i in range(k + 1, NT):
            B, Y = F[blk[i], K], C[blk[i]]
            for c in range(nk):
                r = piv[i, k, c]
                if r >= 0:
                    tmp = X[c, :].copy()
                    X[c, :] = Y[r, :]
                    Y[r, :] = tmp
                Y -= np.outer(B[:, c], X[c, :])
    return C


def back_substitute(F, Y):
    """U X = Y with U the upper triangle of F, row by row from the bottom."""
    n = F.shape[0]
    X = np.array(Y, dtype=np.float64, copy=True)
    for r in range(n - 1, -1, -1):
        X[r] = (X[r] - F[r, r + 1:] @ X[r + 1:]) / F[r, r]
    return X


def lu_solve(F, piv, nb, B):
    """A X = B from the factors."""
    return back_substitute(F, apply_incpiv(F, piv, nb, B))


def lu_flops(n):
    """Credited work of an order-n LU: 2 n^3 / 3."""
    return 2.0 * n ** 3 / 3.0
