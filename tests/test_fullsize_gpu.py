"""Parity at the benchmark's full size (FP64, N = 10000, the tuned (NB, IB)
and ticket order that bench.py times), through properties the CPU can check
entry by entry: R^T R = A^T A on sampled entries (invariant to R's row
signs, independent of Q), Q^T a_j = r_j on sampled columns through the
separate Q-application kernel, and Q^T (A Z) = R Z with Q^T applied on the
CPU from the stored reflectors and T factors (oracle/tile_apply.py); and,
marked slow, |R| itself against the oracle's unblocked Householder R of the
same matrix up to row signs, at 1e-10 relative."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1102_5328_gb300 import inputs  # noqa: E402

U = 2.0 ** -53
N = 10000
SEED = 10000  # the benchmark's matrix


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1102_5328_gb300 as q
    q.lib()
    return q


@pytest.fixture(scope="module")
def fact(q):
    A = inputs.uniform_matrix(N, N, seed=SEED)
    nb, ib = q.qr_lookup(N, N, torch.float64)
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    f = q.qr_factor(Ad, nb, ib)
    torch.cuda.synchronize()
    return A, f, nb, ib


def test_bench_size_factorization_properties(q, fact):
    A, f, nb, ib = fact
    assert f.status() == 0
    rng = np.random.default_rng(1)
    cn = np.linalg.norm(A, axis=0)

    def rcol(j):
        return f.A[: j + 1, j].cpu().numpy()

    # R^T R = A^T A: |(R^T R - A^T A)_ij| <= 10 n u ||a_i|| ||a_j|| (backward stability)
    for i, j in rng.integers(0, N, size=(48, 2)):
        ri, rj = rcol(int(i)), rcol(int(j))
        k = min(i, j) + 1
        lhs = float(ri[:k] @ rj[:k])
        rhs = float(A[:, i] @ A[:, j])
        assert abs(lhs - rhs) <= 10 * N * U * cn[i] * cn[j], (i, j, lhs, rhs)
    # diagonal entries: ||r_j|| = ||a_j||
    for j in rng.integers(0, N, size=16):
        assert abs(np.linalg.norm(rcol(int(j))) - cn[j]) <= 10 * N * U * cn[j]
    # Q^T a_j = r_j through the Q application (persistent apply kernel)
    cols = rng.choice(N, 8, replace=False)
    C = torch.from_numpy(np.ascontiguousarray(A[:, cols].T)).cuda().t()
    q.qr_apply_qt(f, C, trans=True)
    QtA = C.cpu().numpy()
    for c, j in enumerate(cols):
        r = np.zeros(N)
        r[: j + 1] = rcol(int(j))
        assert np.linalg.norm(QtA[:, c] - r) <= 10 * N * U * cn[j], j


def test_bench_size_stored_factors_applied_on_cpu(q, fact):
    """The stored tile factors (reflectors in A, T blocks) define an
    orthogonal Q with Q^T A = R: applied on the CPU to A Z for random Z."""
    from oracle.tile_apply import tile_qt_apply
    A, f, nb, ib = fact
    F = f.A.cpu().numpy()
    T = f.T.cpu().numpy()
    Z = np.random.default_rng(2).standard_normal((N, 3))
    QtAZ = tile_qt_apply(F, T, nb, ib, A @ Z)
    RZ = np.triu(F) @ Z
    err = np.linalg.norm(QtAZ - RZ) / (np.linalg.norm(A) * np.linalg.norm(Z))
    assert err <= 10 * N * U, err


@pytest.mark.slow
def test_bench_size_r_matches_oracle(q, fact):
    """||D R_gpu - R_oracle||_F / ||R_oracle||_F <= 1e-10, D = diag(+-1) from
    the diagonal signs: the |R| agreement criterion at the benchmark's size
    (the oracle's dgeqr2-style QR of the same N = 10000 matrix)."""
    import oracle
    A, f, nb, ib = fact
    F, _ = oracle.geqr2(A)
    R_or = np.triu(F)
    del F
    R = np.triu(f.A.cpu().numpy())
    D = oracle.row_signs(R, R_or)
    rel = np.linalg.norm(D[:, None] * R - R_or) / np.linalg.norm(R_or)
    assert rel <= 1e-10, rel
