"""Q^T of a flat-tree tile QR applied on the CPU from its stored factors --
TEST INFRASTRUCTURE ONLY (imported by ``tests/`` alone).

A large-N probe: the GPU's factored matrix (reflectors below R, in place)
and its T factors are read back, and Q^T is applied to a few vectors here,
in NumPy, following the tile QR's order of eliminations (Sec. 2.1 of the
paper, flat tree): for each panel k, first the diagonal tile's reflectors
(GEQRT), then, for every tile row i > k in increasing order, the reflectors
that eliminated tile (i, k) against the triangle of tile (k, k) (TSQRT).
Each group of up to IB reflectors is applied as a compact-WY block,
z <- (I - V T V^T)^T z = z - V (T^T (V^T z)), with V of a diagonal tile
unit lower trapezoidal (1 on the diagonal, zeros above) and V of an
eliminated tile [e-rows of tile k; the full tile i].

Storage read (the library's documented layout): the factored matrix is
column-major m x n; T holds an IB x NB block per tile (i, k) at offset
(k * MT + i) * IB * NB, inner block l's ib x ib upper triangle at columns
l * IB ... (leading dimension IB).

Nothing here is shared with the GPU path; it only reads the arrays.
"""
import numpy as np


def tile_qt_apply(F, T, nb, ib, Z):
    """Q^T Z for the flat-tree tile QR factors (F: m x n factored matrix,
    T: flat array of the block factors, Z: m x k). Returns a new array."""
    F = np.asarray(F, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64).reshape(-1)
    Z = np.array(Z, dtype=np.float64, copy=True)
    if Z.ndim == 1:
        Z = Z[:, None]
    m, n = F.shape
    MT, NT = -(-m // nb), -(-n // nb)

    def tblock(i, k, l0, w):
        base = (k * MT + i) * ib * nb
        blk = np.empty((w, w))
        for p in range(w):
            col = T[base + (l0 + p) * ib: base + (l0 + p) * ib + w]
            blk[:, p] = col
        return np.triu(blk)

    for k in range(min(MT, NT)):
        r0 = k * nb
        rk = min(nb, m - r0)
        ck = min(nb, n - r0)
        # GEQRT(k): reflectors of the diagonal tile
        for l0 in range(0, ck, ib):
            w = min(ib, ck - l0)
            V = np.array(F[r0:r0 + rk, r0 + l0:r0 + l0 + w], copy=True)
            for p in range(w):
                V[: l0 + p, p] = 0.0
                V[l0 + p, p] = 1.0
            Tl = tblock(k, k, l0, w)
            zk = Z[r0:r0 + rk]
            W = Tl.T @ (V.T @ zk)
            Z[r0:r0 + rk] = zk - V @ W
        # TSQRT(i, k), i = k+1 ..: reflectors [e_(l0+p) in tile k; V(:, p) in tile i]
        for i in range(k + 1, MT):
            s0 = i * nb
            ri = min(nb, m - s0)
            for l0 in range(0, ck, ib):
                w = min(ib, ck - l0)
                V = F[s0:s0 + ri, r0 + l0:r0 + l0 + w]
                Tl = tblock(i, k, l0, w)
                top = Z[r0 + l0:r0 + l0 + w]
                W = Tl.T @ (top + V.T @ Z[s0:s0 + ri])
                Z[r0 + l0:r0 + l0 + w] = top - W
                Z[s0:s0 + ri] = Z[s0:s0 + ri] - V @ W
    return Z


def t_factor(V, tau):
    """T of a block of reflectors with V's columns as given and scalars tau,
    by the columnwise forward recurrence T(p,p) = tau_p,
    T(0:p, p) = -tau_p T(0:p, 0:p) (V^T v_p)(0:p)."""
    w = len(tau)
    Tm = np.zeros((w, w))
    G = V.T @ V
    for p in range(w):
        Tm[p, p] = tau[p]
        if p:
            Tm[:p, p] = -tau[p] * (Tm[:p, :p] @ G[:p, p])
    return Tm
