"""GPU parity of the tile QR (C ABI: qr_factor_d, qr_apply_qt_d) against the
CPU oracle: backward error, orthogonality, |R| up to row signs, exact sign
agreement on a single tile, determinism, and host-made faults."""
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


def to_dev(x):
    """Column-major CUDA copy of a NumPy matrix."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x).T)).cuda().t()


def _gpu_factor(q, A_np, nb, ib):
    A = to_dev(A_np)
    t_elems, _ = q.qr_workspace(A.shape[0], A.shape[1], nb, ib, A.dtype)
    T = torch.zeros(max(t_elems, 1), dtype=A.dtype, device="cuda")  # unused slots stay zero
    f = q.qr_factor(A, nb, ib, T=T)
    torch.cuda.synchronize()
    return f


def _check(q, A_np, nb, ib, r_tol=1e-10):
    m, n = A_np.shape
    f = _gpu_factor(q, A_np, nb, ib)
    assert f.status() == 0
    R = np.triu(f.A[:n].cpu().numpy())
    Q = q.form_q(f).cpu().numpy()
    torch.cuda.synchronize()
    res = oracle.fact_residual(A_np, Q, R) / (n * U)
    orth = oracle.orth_residual(Q) / (n * U)
    assert res <= 10.0, res
    assert orth <= 10.0, orth
    F, _ = oracle.geqr2(A_np)
    R_or = np.triu(F[:n])
    D = oracle.row_signs(R, R_or)
    rel = np.linalg.norm(D[:, None] * R - R_or) / np.linalg.norm(R_or)
    assert rel <= r_tol, rel
    return f, R, R_or


def test_single_tile_matches_oracle_signs(q):
    """NB >= max(m, n): tile QR is one GEQRT, the blocked Householder QR with
    the oracle's sign convention, so R and the reflectors match directly."""
    A = inputs.uniform_matrix(128, 128, seed=3)
    f, R, R_or = _check(q, A, 128, 32)
    assert np.array_equal(np.sign(np.diag(R)), np.sign(np.diag(R_or)))
    assert np.abs(R - R_or).max() <= 1e-13 * np.abs(R_or).max()
    F, tau = oracle.geqr2(A)
    V = np.tril(f.A.cpu().numpy(), -1)
    assert np.abs(V - np.tril(F, -1)).max() < 1e-12
    # T's diagonal holds tau (IB x NB block factors, ld IB)
    T = f.T[: 32 * 128].cpu().numpy().reshape(128, 32).T
    taus = np.array([T[p % 32, p] for p in range(128)])
    assert np.abs(taus - tau).max() < 1e-13


@pytest.mark.parametrize("m,n,nb,ib", [
    (512, 512, 128, 32),    # the 512 x 512, NB = 128, IB = 32 case
    (300, 200, 64, 16),
    (1000, 1000, 96, 32),   # NB does not divide N: ragged edge tiles
    (700, 300, 128, 9),     # odd IB, ragged inner blocks
    (513, 513, 256, 128),   # IB > 32: level-2 sub-panels inside a block
    (640, 600, 512, 256),   # largest IB, split update tasks
    (450, 450, 160, 80),
    (257, 129, 32, 8),
    (64, 64, 64, 32),
    (100, 1, 32, 8),        # a single column
    (33, 33, 8, 8),
])
def test_factor_parity(q, m, n, nb, ib):
    A = inputs.uniform_matrix(m, n, seed=m * 7 + n)
    _check(q, A, nb, ib)


def test_apply_qt_is_transpose(q):
    m, n = 400, 300
    A = inputs.uniform_matrix(m, n, seed=9)
    f = _gpu_factor(q, A, 64, 16)
    C = to_dev(inputs.normal_matrix(m, 5, seed=2))
    C0 = C.clone()
    q.qr_apply_qt(f, C, trans=True)
    # Q^T A = [R; 0]
    Ad = to_dev(A)
    q.qr_apply_qt(f, Ad, trans=True)
    R = torch.triu(f.A[:n]).cpu().numpy()
    QtA = Ad.cpu().numpy()
    assert np.abs(QtA[:n] - R).max() < 50 * n * U
    assert np.abs(QtA[n:]).max() < 50 * n * U
    q.qr_apply_qt(f, C, trans=False)
    assert torch.allclose(C, C0, atol=100 * n * U, rtol=0)
    # the column-chunk kernel and the dependency-ordered persistent kernel
    # perform the same operations per column: identical results
    for trans in (True, False):
        C1 = to_dev(inputs.normal_matrix(m, 70, seed=3))
        C2 = C1.clone().t().contiguous().t()
        q.qr_apply_qt(f, C1, trans=trans, parallel=False)
        q.qr_apply_qt(f, C2, trans=trans, parallel=True)
        assert torch.equal(C1, C2)


def test_deterministic_and_schedule_independent(q):
    """The DAG fixes every tile's operation sequence, so the result is bitwise
    identical run to run and with one CTA running the tasks sequentially."""
    A = inputs.uniform_matrix(777, 600, seed=4)
    f1 = _gpu_factor(q, A, 96, 24)
    f2 = _gpu_factor(q, A, 96, 24)
    assert torch.equal(f1.A, f2.A) and torch.equal(f1.T, f2.T)
    q.qr_set_option(q.QR_OPT_GRID_LIMIT, 1)
    try:
        f3 = _gpu_factor(q, A, 96, 24)
    finally:
        q.qr_set_option(q.QR_OPT_GRID_LIMIT, 0)
    assert torch.equal(f1.A, f3.A) and torch.equal(f1.T, f3.T)


def test_missing_task_times_out_with_status(q):
    """Host-made fault: drop one task from the list; its dependents' bounded
    waits expire, the kernel returns, the status word says so, and the
    context stays usable."""
    A = inputs.uniform_matrix(256, 256, seed=5)
    q.qr_set_option(q.QR_OPT_WAIT_TIMEOUT_US, 200_000)
    q.qr_set_option(q.QR_OPT_DROP_TASK, 3)
    try:
        f = _gpu_factor(q, A, 64, 16)
        st = f.status()
    finally:
        q.qr_set_option(q.QR_OPT_DROP_TASK, -1)
        q.qr_set_option(q.QR_OPT_WAIT_TIMEOUT_US, 20_000_000)
    assert st & q.QR_DEV_TIMEOUT
    _check(q, A, 64, 16)


def test_nonfinite_input_flagged(q):
    A = inputs.uniform_matrix(128, 128, seed=6)
    A[5, 0] = np.nan
    f = _gpu_factor(q, A, 64, 16)
    assert f.status() & q.QR_DEV_NONFINITE


def test_invalid_arguments_rejected(q):
    A = q.colmajor_empty(100, 50, torch.float64)
    lib = q.lib()
    import ctypes
    assert lib.qr_factor_d(100, 50, ctypes.c_void_p(A.data_ptr()), 99, 32, 8, None, None, 0, None) == -4
    assert lib.qr_factor_d(100, 50, ctypes.c_void_p(A.data_ptr()), 100, 600, 8, None, None, 0, None) == -5
    assert lib.qr_factor_d(100, 50, ctypes.c_void_p(A.data_ptr()), 100, 32, 33, None, None, 0, None) == -6
    assert lib.qr_factor_d(50, 100, ctypes.c_void_p(A.data_ptr()), 100, 32, 8, None, None, 0, None) == -2


def test_double_buffered_staging_is_bitwise_neutral(q):
    """The TS-mode update double-buffers its reflector staging only when the
    reflector array has an even leading dimension; the arithmetic is the same
    either way, so applying Q^T from a copy of the factors with an odd
    leading dimension must give bitwise the same result."""
    m, n = 400, 300
    A = inputs.uniform_matrix(m, n, seed=21)
    f = _gpu_factor(q, A, 64, 16)
    A_odd_store = torch.zeros((n, m + 1), dtype=torch.float64, device="cuda")
    A_odd = A_odd_store.t()[:m]  # column-major view, lda = m + 1 (odd)
    A_odd.copy_(f.A)
    f_odd = q.Factorization(A_odd, f.T, None, f.nb, f.ib)
    for trans in (True, False):
        C1 = to_dev(inputs.normal_matrix(m, 40, seed=8))
        C2 = C1.clone().t().contiguous().t()
        q.qr_apply_qt(f, C1, trans=trans)
        q.qr_apply_qt(f_odd, C2, trans=trans)
        assert torch.equal(C1, C2)


@pytest.mark.parametrize("nrhs", [1, 3, 8, 16])
def test_narrow_application_matches_wide(q, nrhs):
    """Few right-hand sides take the shared-memory narrow path in the
    dependency-ordered application; the column-chunk kernel takes the wide
    path. Same operations, different summation order: equal to rounding."""
    m, n = 640, 384
    A = inputs.uniform_matrix(m, n, seed=31)
    f = _gpu_factor(q, A, 64, 8)
    for trans in (True, False):
        C1 = to_dev(inputs.normal_matrix(m, nrhs, seed=nrhs))
        C2 = C1.clone().t().contiguous().t()
        q.qr_apply_qt(f, C1, trans=trans, parallel=False)
        q.qr_apply_qt(f, C2, trans=trans, parallel=True)
        assert torch.allclose(C1, C2, rtol=0, atol=100 * n * U * float(C1.abs().max()))


def test_task_trace(q):
    """qr_set_trace: one record per task of the persistent factorization,
    timestamps ordered, SM ids within the device, tracing off afterwards."""
    m, n, nb, ib = 700, 500, 64, 16
    A = torch.from_numpy(np.ascontiguousarray(inputs.uniform_matrix(m, n, seed=3).T)).cuda().t()
    ntasks = q.qr_task_count(m, n, nb, ib)
    buf = torch.full((ntasks + 8, 4), -1, dtype=torch.int64, device="cuda")
    q.qr_set_trace(buf)
    try:
        q.qr_factor(A, nb, ib)
        torch.cuda.synchronize()
    finally:
        q.qr_set_trace(None)
    task, typ, sm, t_take, t_ready, t_done = q.read_trace(buf, ntasks)
    assert sorted(task.tolist()) == list(range(ntasks))
    assert set(typ.tolist()) == {0, 1, 2, 3}
    assert np.all(t_take <= t_ready) and np.all(t_ready <= t_done)
    assert sm.max() < torch.cuda.get_device_properties(0).multi_processor_count
    assert np.all(buf[ntasks:].cpu().numpy() == -1)


def test_ticket_order_weights_are_bitwise_neutral(q):
    """Measured task costs and the flop-weight options only reorder the
    tickets: the factorization is bitwise the same under every order."""
    A = inputs.uniform_matrix(900, 700, seed=6)
    q.qr_set_task_costs(torch.float64, 64, 8, None)
    f1 = _gpu_factor(q, A, 64, 8)
    q.qr_set_task_costs(torch.float64, 64, 8, [9.0, 1.0, 7.0, 2.0])
    try:
        f2 = _gpu_factor(q, A, 64, 8)
    finally:
        q.qr_set_task_costs(torch.float64, 64, 8, None)
    q.qr_set_option(q.QR_OPT_PANEL_WEIGHT, 500)
    q.qr_set_option(q.QR_OPT_UNMQR_WEIGHT, 20)
    try:
        f3 = _gpu_factor(q, A, 64, 8)
    finally:
        q.qr_set_option(q.QR_OPT_PANEL_WEIGHT, 150)
        q.qr_set_option(q.QR_OPT_UNMQR_WEIGHT, 100)
    assert torch.equal(f1.A, f2.A) and torch.equal(f1.T, f2.T)
    assert torch.equal(f1.A, f3.A) and torch.equal(f1.T, f3.T)


def test_calibration_measures_every_task_type(q):
    """calibrate.measure on a small order: one positive median service time
    per task type, task counts matching the flat tree's DAG, and a report
    whose busy fractions lie in [0, 1]."""
    from paper_1102_5328_gb300 import calibrate
    n, nb, ib = 640, 64, 16
    costs, counts, span_ms = calibrate.measure(n, nb, ib, torch.float64)
    nt = n // nb
    assert counts == [nt, nt * (nt - 1) // 2, nt * (nt - 1) // 2, sum(k * k for k in range(nt))]
    assert all(c > 0 for c in costs) and span_ms > 0
    rep = calibrate.report(n, nb, ib, torch.float64, 2 * torch.cuda.get_device_properties(0).multi_processor_count)
    assert all(0.0 <= b <= 1.0 + 1e-9 for b in rep["busy_per_tenth"])
    assert [t["count"] for t in rep["types"]] == counts


@pytest.mark.parametrize("m,n,nb,ib", [(777, 600, 96, 24), (1024, 1024, 128, 16), (333, 300, 64, 16)])
def test_factor_fp32_flat_tree_budget(q, m, n, nb, ib):
    """FP32 flat-tree factorization (the FP32 update path with 16-byte shared
    loads): R agrees with the oracle's QR of the FP32-rounded input, up to
    row signs, within 10 n u_32, and Q^T A reproduces R to the same budget."""
    A = inputs.uniform_matrix(m, n, seed=m + 3 * n)
    A32 = A.astype(np.float32).astype(np.float64)
    def dev32(x):
        return torch.from_numpy(np.ascontiguousarray(x.T).astype(np.float32)).cuda().t()

    f = q.qr_factor(dev32(A), nb, ib, p=1)
    torch.cuda.synchronize()
    R = np.triu(f.A[:n].double().cpu().numpy())
    F, _ = oracle.geqr2(A32)
    R_or = np.triu(F[:n])
    D = oracle.row_signs(R, R_or)
    u32 = 2.0 ** -24
    assert np.linalg.norm(D[:, None] * R - R_or) / np.linalg.norm(R_or) <= 10 * n * u32
    C = dev32(A)
    q.qr_apply_qt(f, C, trans=True)
    QtA = C.double().cpu().numpy()
    assert np.linalg.norm(np.triu(QtA[:n]) - R) / np.linalg.norm(R) <= 10 * n * u32
    if m > n:
        assert np.linalg.norm(QtA[n:]) / np.linalg.norm(R) <= 10 * n * u32


@pytest.mark.parametrize("m,n,nb,ib", [(777, 600, 96, 24), (1000, 1000, 128, 8), (513, 300, 64, 7)])
def test_stored_factors_applied_on_cpu(q, m, n, nb, ib):
    """The GPU's stored factors (reflectors below R, T blocks), applied on
    the CPU by an independent restatement of the tile updates
    (oracle/tile_apply.py), take A to R over several panels and ragged
    tiles; NB = 128 runs the FP64 update tasks as two column chunks."""
    from oracle.tile_apply import tile_qt_apply
    A = inputs.uniform_matrix(m, n, seed=m + 11 * n)
    f = _gpu_factor(q, A, nb, ib)
    F = f.A.cpu().numpy()
    T = f.T.cpu().numpy()
    QtA = tile_qt_apply(F, T, nb, ib, A)
    R = np.triu(F[:n])
    assert np.linalg.norm(QtA[:n] - R) / np.linalg.norm(R) <= 10 * n * 2.0 ** -53
    if m > n:
        assert np.linalg.norm(QtA[n:]) / np.linalg.norm(R) <= 10 * n * 2.0 ** -53
