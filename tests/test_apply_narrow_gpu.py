"""The Q application on a few columns (qr_apply_qt_p_*, the least-squares
refinement's Q^T r and Q d, whose tasks stage a whole reflector tile and
C's rows in shared memory) against the oracle and the factorization itself.

For every shape (flat tree p = 1 and binary-tree domains p > 1, ragged tile
rows and columns, IB that does not divide NB, 1..16 columns):
  * Q^T A[:, cols] = R[:, cols] on top, zero below (the defining property of
    the factors, Sec. 2.1), within 50 n u;
  * the top n rows of Q^T C equal D Q_o^T C with Q_o the oracle's Householder
    QR of the same matrix and D its row signs (1e-9 of ||C||);
  * Q^T keeps column norms, and Q (Q^T C) = C, within 50 n u ||C||.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1102_5328_gb300 import inputs  # noqa: E402

U64 = 2.0 ** -53
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1102_5328_gb300 as q
    q.lib()
    return q


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).to(dtype).cuda().t()


def _apply(q, f, C, trans):
    """qr_apply_qt_p_* through the C ABI, p = 1 included."""
    m, n = f.m, f.n
    nrhs = C.shape[1]
    wb = ctypes.c_int64()
    L = q.lib()
    assert L.qr_apply_workspace_p(m, n, nrhs, f.nb, f.p, ctypes.byref(wb)) == 0
    ws = torch.empty(wb.value, dtype=torch.uint8, device="cuda")
    fn = L.qr_apply_qt_p_d if C.dtype == torch.float64 else L.qr_apply_qt_p_s
    lda = f.A.stride(1) if n > 1 else m
    ldc = C.stride(1) if nrhs > 1 else m  # a one-column tensor's stride(1) is 1
    rc = fn(m, n, nrhs, ctypes.c_void_p(f.A.data_ptr()), lda, f.nb, f.ib, f.p, ctypes.c_void_p(f.T.data_ptr()),
            ctypes.c_void_p(C.data_ptr()), ldc, 1 if trans else 0, ctypes.c_void_p(ws.data_ptr()), wb.value, None)
    torch.cuda.synchronize()
    assert rc == 0
    return C


def _factor(q, A, nb, ib, p, dtype):
    m, n = A.shape
    tel, _ = q.qr_workspace_p(m, n, nb, ib, p, dtype)
    T = torch.zeros(max(tel, 1), dtype=dtype, device="cuda")
    f = q.qr_factor(_dev(A, dtype), nb, ib, T=T, p=p)
    torch.cuda.synchronize()
    assert f.status() == 0
    return f


CASES = [
    (1000, 300, 64, 16, 1, 8),
    (1000, 300, 64, 16, 4, 8),
    (777, 500, 48, 9, 2, 5),      # ragged tiles, IB not dividing NB
    (2048, 256, 64, 32, 8, 8),    # IB = 32
    (513, 129, 32, 8, 5, 16),     # short last tile row, 16 columns
    (300, 300, 64, 8, 1, 1),      # square, one column
    (4096, 64, 64, 16, 16, 3),    # one tile column, 64 tile rows
]


@pytest.mark.parametrize("m,n,nb,ib,p,k", CASES)
def test_narrow_apply_fp64(q, m, n, nb, ib, p, k):
    A = inputs.uniform_matrix(m, n, seed=m + 7 * n + p)
    f = _factor(q, A, nb, ib, p, torch.float64)
    R = np.triu(f.A[:n].cpu().numpy())
    cols = np.linspace(0, n - 1, k).astype(int)
    # Q^T A[:, cols] = [R[:, cols]; 0]
    out = _apply(q, f, _dev(A[:, cols], torch.float64), True).cpu().numpy()
    assert np.abs(out[:n] - R[:, cols]).max() < 50 * n * U64
    if m > n:
        assert np.abs(out[n:]).max() < 50 * n * U64
    # against the oracle's Q on a random C
    G = np.random.default_rng(m + n + k).standard_normal((m, k))
    F, tau = oracle.geqr2(A)
    D = oracle.row_signs(R, np.triu(F[:n]))
    ref = oracle.apply_qt(F, tau, G.copy())
    got = _apply(q, f, _dev(G, torch.float64), True).cpu().numpy()
    assert np.linalg.norm(D[:, None] * got[:n] - ref[:n]) <= 1e-9 * np.linalg.norm(G)
    assert np.allclose(np.linalg.norm(got, axis=0), np.linalg.norm(G, axis=0), rtol=50 * n * U64)
    # Q (Q^T G) = G
    back = _apply(q, f, _dev(got, torch.float64), False).cpu().numpy()
    assert np.abs(back - G).max() <= 50 * n * U64 * np.abs(G).max()


@pytest.mark.parametrize("m,n,nb,ib,p,k", [(1000, 300, 64, 16, 2, 8), (777, 500, 48, 9, 1, 5),
                                           (2048, 256, 64, 32, 4, 16)])
def test_narrow_apply_fp32(q, m, n, nb, ib, p, k):
    A = inputs.uniform_matrix(m, n, seed=m + n + 11)
    f = _factor(q, A, nb, ib, p, torch.float32)
    G = np.random.default_rng(k).standard_normal((m, k))
    got = _apply(q, f, _dev(G, torch.float32), True).double().cpu().numpy()
    assert np.allclose(np.linalg.norm(got, axis=0), np.linalg.norm(G, axis=0), rtol=50 * n * U32)
    back = _apply(q, f, _dev(got, torch.float32), False).double().cpu().numpy()
    assert np.abs(back - G).max() <= 50 * n * U32 * np.abs(G).max()
