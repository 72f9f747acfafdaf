"""Pins of the CPU tile-Q applier (oracle/tile_apply.py) against the
unblocked oracle alone: tile factors assembled from oracle.geqr2 runs --
one diagonal tile, then a triangle stacked on a second tile -- must give
the same Q^T as the unblocked Householder products."""
import numpy as np
import pytest

import oracle
from oracle.tile_apply import t_factor, tile_qt_apply
from paper_1102_5328_gb300 import inputs


def _t_layout(blocks, MT, nb, ib, entries):
    """Flat T array: for tile (i, k), block l at columns l*ib (ld ib)."""
    NT = 1
    T = np.full(MT * NT * ib * nb, np.nan)
    for (i, k), blist in entries.items():
        base = (k * MT + i) * ib * nb
        for l0, Tl in blist:
            w = Tl.shape[0]
            for p in range(w):
                T[base + (l0 + p) * ib: base + (l0 + p) * ib + w] = Tl[:, p]
    return T


def _ge_blocks(F, tau, ib):
    rk, ck = F.shape[0], len(tau)
    out = []
    for l0 in range(0, ck, ib):
        w = min(ib, ck - l0)
        V = np.array(F[:, l0:l0 + w], copy=True)
        for p in range(w):
            V[: l0 + p, p] = 0.0
            V[l0 + p, p] = 1.0
        out.append((l0, t_factor(V, tau[l0:l0 + w])))
    return out


@pytest.mark.parametrize("m,n,nb,ib", [(40, 40, 48, 8), (37, 30, 40, 7), (20, 20, 20, 20)])
def test_single_tile_matches_unblocked(m, n, nb, ib):
    A = inputs.uniform_matrix(m, n, seed=m * n)
    F, tau = oracle.geqr2(A)
    T = _t_layout(None, 1, nb, ib, {(0, 0): _ge_blocks(F, tau, ib)})
    Z = inputs.normal_matrix(m, 3, seed=1)
    got = tile_qt_apply(F, T, nb, ib, Z)
    ref = oracle.apply_qt(F, tau, Z.copy())
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("nb,ib,short", [(16, 4, 0), (16, 5, 5), (12, 12, 3)])
def test_triangle_on_tile_matches_unblocked(nb, ib, short):
    """GEQRT of tile 0, then TSQRT of [R0; tile 1] (tile 1 possibly short)."""
    m = 2 * nb - short
    A = inputs.uniform_matrix(m, nb, seed=nb + short)
    F0, tau0 = oracle.geqr2(A[:nb])
    R0 = np.triu(F0)
    S = np.vstack([R0, A[nb:]])
    Fs, taus = oracle.geqr2(S)
    # the stacked reflectors are e_p on the triangle (exact zeros below it)
    assert np.all(np.tril(Fs[:nb], -1) == 0.0)
    Ft = np.vstack([np.triu(Fs[:nb]) + np.tril(F0, -1), Fs[nb:]])
    ts_blocks = []
    for l0 in range(0, nb, ib):
        w = min(ib, nb - l0)
        ts_blocks.append((l0, t_factor(Fs[nb:, l0:l0 + w], taus[l0:l0 + w])))
    T = _t_layout(None, 2, nb, ib, {(0, 0): _ge_blocks(F0, tau0, ib), (1, 0): ts_blocks})
    Z = inputs.normal_matrix(m, 2, seed=2)
    got = tile_qt_apply(Ft, T, nb, ib, Z)
    Y = Z.copy()
    Y[:nb] = oracle.apply_qt(F0, tau0, Y[:nb].copy())
    ref = oracle.apply_qt(Fs, taus, Y)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    # and Q^T A is the stacked R
    QtA = tile_qt_apply(Ft, T, nb, ib, A)
    assert np.abs(QtA[:nb] - np.triu(Fs[:nb])).max() <= 1e-13 * np.abs(Fs[:nb]).max()
    assert np.abs(QtA[nb:]).max() <= 1e-13 * np.abs(Fs[:nb]).max()


def test_flat_tree_order_over_three_tile_rows():
    """GEQRT(0), TSQRT(1, 0), TSQRT(2, 0): the second elimination works on
    the triangle the first one left, so the order of the TS steps matters."""
    nb, ib = 12, 5
    A = inputs.uniform_matrix(3 * nb, nb, seed=33)
    F0, tau0 = oracle.geqr2(A[:nb])
    Fs1, taus1 = oracle.geqr2(np.vstack([np.triu(F0), A[nb:2 * nb]]))
    Fs2, taus2 = oracle.geqr2(np.vstack([np.triu(Fs1[:nb]), A[2 * nb:]]))
    Ft = np.vstack([np.triu(Fs2[:nb]) + np.tril(F0, -1), Fs1[nb:], Fs2[nb:]])

    def ts(Fs, taus):
        return [(l0, t_factor(Fs[nb:, l0:l0 + min(ib, nb - l0)], taus[l0:l0 + min(ib, nb - l0)]))
                for l0 in range(0, nb, ib)]

    T = _t_layout(None, 3, nb, ib, {(0, 0): _ge_blocks(F0, tau0, ib), (1, 0): ts(Fs1, taus1),
                                    (2, 0): ts(Fs2, taus2)})
    Z = inputs.normal_matrix(3 * nb, 2, seed=3)
    got = tile_qt_apply(Ft, T, nb, ib, Z)
    Y = Z.copy()
    Y[:nb] = oracle.apply_qt(F0, tau0, Y[:nb].copy())
    Y[:2 * nb] = oracle.apply_qt(Fs1, taus1, Y[:2 * nb].copy())
    Y[np.r_[0:nb, 2 * nb:3 * nb]] = oracle.apply_qt(Fs2, taus2, Y[np.r_[0:nb, 2 * nb:3 * nb]].copy())
    assert np.abs(got - Y).max() <= 1e-13 * np.abs(Y).max()
