"""Tile QR with p panel domains merged by a binary tree (TTQRT/TTMQR; the
paper's communication-avoiding variant for tall-skinny matrices) against the
CPU oracle, and p = 1 against the flat-tree entry point."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1102_5328_gb300 import inputs

U = 2.0 ** -53


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1102_5328_gb300 as q
    q.lib()
    return q


def to_dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).to(dtype).cuda().t()


@pytest.mark.parametrize("m,n,nb,ib,p", [
    (1024, 256, 64, 16, 4),     # tall-skinny, 16 x 4 tiles
    (2000, 300, 64, 8, 3),      # ragged in both directions, uneven domains
    (777, 777, 96, 24, 2),      # square, ragged
    (1300, 200, 128, 32, 8),    # more domains than some steps have rows
    (4096, 64, 64, 16, 16),     # one tile column, 64 tile rows
    (513, 129, 32, 8, 5),       # ragged last tile row shorter than the panel
    (640, 600, 256, 128, 2),    # split update tasks, IB > 32 sub-panels
])
def test_tree_parity(q, m, n, nb, ib, p):
    A = inputs.uniform_matrix(m, n, seed=m + n + p)
    Ad = to_dev(A)
    f = q.qr_factor(Ad, nb, ib, p=p)
    torch.cuda.synchronize()
    assert f.status() == 0
    R = np.triu(f.A[:n].cpu().numpy())
    Q = q.form_q(f).cpu().numpy()
    assert oracle.fact_residual(A, Q, R) / (n * U) <= 10
    assert oracle.orth_residual(Q) / (n * U) <= 10
    F, _ = oracle.geqr2(A)
    R_or = np.triu(F[:n])
    D = oracle.row_signs(R, R_or)
    assert np.linalg.norm(D[:, None] * R - R_or) / np.linalg.norm(R_or) <= 1e-10
    # Q^T A = [R; 0]
    C = to_dev(A)
    q.qr_apply_qt(f, C, trans=True)
    QtA = C.cpu().numpy()
    assert np.abs(QtA[:n] - R).max() < 50 * n * U
    if m > n:
        assert np.abs(QtA[n:]).max() < 50 * n * U


def test_one_domain_is_the_flat_tree(q):
    A = inputs.uniform_matrix(700, 500, seed=3)
    f1 = q.qr_factor(to_dev(A), 64, 16)
    T = torch.zeros(q.qr_workspace_p(700, 500, 64, 16, 1)[0], dtype=torch.float64, device="cuda")
    fp = q.qr_factor(to_dev(A), 64, 16, T=T, p=2)  # warm the p path
    A1 = to_dev(A)
    tel, sb = q.qr_workspace_p(700, 500, 64, 16, 1)
    Tp = torch.zeros(tel, dtype=torch.float64, device="cuda")
    scr = torch.empty(sb, dtype=torch.uint8, device="cuda")
    import ctypes
    L = q.lib()
    assert L.qr_factor_p_d(700, 500, ctypes.c_void_p(A1.data_ptr()), 700, 64, 16, 1, ctypes.c_void_p(Tp.data_ptr()),
                           ctypes.c_void_p(scr.data_ptr()), sb, None) == 0
    torch.cuda.synchronize()
    assert torch.equal(A1, f1.A)
    assert fp.status() == 0


def test_tree_fp32_budget(q):
    m, n = 2048, 256
    A = inputs.uniform_matrix(m, n, seed=8)
    f = q.qr_factor(to_dev(A, torch.float32), 64, 16, p=4)
    R = np.triu(f.A[:n].double().cpu().numpy())
    F, _ = oracle.geqr2(A.astype(np.float32).astype(np.float64))
    R_or = np.triu(F[:n])
    D = oracle.row_signs(R, R_or)
    assert np.linalg.norm(D[:, None] * R - R_or) / np.linalg.norm(R_or) <= 10 * n * 2.0 ** -24
