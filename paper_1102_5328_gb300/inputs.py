"""Seeded synthetic inputs shared by the GPU path's tests/benchmark and the
oracle's tests. Random numbers only: this module holds none of the QR
method's arithmetic.

Every generator uses NumPy's PCG64 ``default_rng(seed)`` and returns
column-major (Fortran-ordered) arrays, so both sides see identical bytes.

Workload shapes follow the paper's experiments (matrices of order N,
entries uniform, Sec. 3 and Sec. 6.1: N in {500, 1000, ..., 10000}) and the
extensions this library adds (tall-skinny shapes, batches of small uneven
matrices, conditioned least-squares problems).
"""
import numpy as np


def uniform_matrix(m, n, seed, dtype=np.float64):
    """m x n, entries i.i.d. uniform[-0.5, 0.5)."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray((rng.random((n, m)).T - 0.5).astype(dtype))


def normal_matrix(m, n, seed, dtype=np.float64):
    """m x n, entries i.i.d. N(0, 1)."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, m)).T.astype(dtype))


def conditioned_matrix(m, n, kappa, seed):
    """A = U diag(sigma) V^T with geometric singular values from 1 down to
    1/kappa. U (m x n) and V (n x n) are the orthonormal factors of seeded
    Gaussian matrices, produced by NumPy's LAPACK QR (input synthesis only)."""
    rng = np.random.default_rng(seed)
    G1 = rng.standard_normal((m, n))
    G2 = rng.standard_normal((n, n))
    U, _ = np.linalg.qr(G1)
    V, _ = np.linalg.qr(G2)
    if n > 1:
        sigma = 10.0 ** (-np.log10(kappa) * np.arange(n) / (n - 1))
    else:
        sigma = np.ones(1)
    return np.asfortranarray((U * sigma) @ V.T)


def spd_matrix(n, seed):
    """Symmetric positive definite n x n: G G^T / n + I with G (n x n) N(0,1)
    from seed (eigenvalues in about [1, 5])."""
    G = normal_matrix(n, n, seed)
    return np.asfortranarray(G @ G.T / n + np.eye(n))


def ls_problem(m, n, nrhs, kappa, seed):
    """(A, B): A from conditioned_matrix(seed), B (m x nrhs) N(0,1) from seed+1."""
    A = conditioned_matrix(m, n, kappa, seed)
    B = normal_matrix(m, nrhs, seed + 1)
    return A, B


def batch_shapes(count, seed, m_lo=32, m_hi=512, n_lo=16):
    """Uneven batch: m ~ U{m_lo..m_hi}, n ~ U{n_lo..m} (both inclusive)."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(m_lo, m_hi + 1, size=count)
    ns = np.array([rng.integers(n_lo, mm + 1) for mm in ms])
    return ms.astype(np.int64), ns.astype(np.int64)


def batch_matrices(ms, ns, seed, dtype=np.float64):
    """One N(0,1) matrix per (m, n), drawn in order from one seeded stream."""
    rng = np.random.default_rng(seed)
    out = []
    for m, n in zip(ms, ns):
        out.append(np.asfortranarray(rng.standard_normal((int(n), int(m))).T.astype(dtype)))
    return out


def mlp_init(seed, layers=((4, 64), (64, 64), (64, 1))):
    """Initial weights of the cost-model MLP: each Linear(in, out) draws
    W (out x in, row-major) and b (out) uniform in [-1/sqrt(in), 1/sqrt(in)]
    from one seeded stream. Returns [W1, b1, W2, b2, W3, b3] as float64."""
    rng = np.random.default_rng(seed)
    out = []
    for fin, fout in layers:
        bound = 1.0 / np.sqrt(fin)
        out.append(rng.uniform(-bound, bound, size=(fout, fin)))
        out.append(rng.uniform(-bound, bound, size=(fout,)))
    return out
