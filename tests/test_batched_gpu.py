"""Batched uneven QR on the GPU (C ABI: qr_batched_plan,
qr_factor_batched_d/_s) against the oracle, matrix by matrix, eager and
replayed from a captured CUDA graph."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle
from paper_1102_5328_gb300 import inputs

U64 = 2.0 ** -53
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1102_5328_gb300 as q
    q.lib()
    return q


def _dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x.T)).to(dtype).cuda().t()


def _batch(count, seed, m_hi=200):
    ms, ns = inputs.batch_shapes(count, seed, m_lo=32, m_hi=m_hi)
    return inputs.batch_matrices(ms, ns, seed + 1)


def _check_fp64(q, plan, mats_np, outs, full=True):
    for b, (A_np, A) in enumerate(zip(mats_np, outs)):
        m, n = A_np.shape
        R = np.triu(A[:n].cpu().numpy())
        F, _ = oracle.geqr2(A_np)
        R_or = np.triu(F[:n])
        D = oracle.row_signs(R, R_or)
        rel = np.linalg.norm(D[:, None] * R - R_or) / np.linalg.norm(R_or)
        assert rel <= 1e-12, (b, rel)
        if full and b % 4 == 0:
            Q = q.form_q(plan.factorization(b, A)).cpu().numpy()
            assert oracle.fact_residual(A_np, Q, R) / (n * U64) <= 10
            assert oracle.orth_residual(Q) / (n * U64) <= 10


@pytest.mark.parametrize("force_nb,force_ib", [(0, 0), (32, 8), (64, 16), (512, 32)])
def test_batched_fp64(q, force_nb, force_ib):
    mats_np = _batch(48, seed=7)
    outs = [_dev(a) for a in mats_np]
    plan = q.BatchedPlan(outs, force_nb, force_ib)
    plan.launch()
    torch.cuda.synchronize()
    assert plan.status() == 0
    _check_fp64(q, plan, mats_np, outs)


def test_batched_fp32_budget(q):
    mats_np = _batch(32, seed=9)
    outs = [_dev(a, torch.float32) for a in mats_np]
    plan = q.BatchedPlan(outs, 64, 16)
    plan.launch()
    torch.cuda.synchronize()
    for A_np, A in zip(mats_np, outs):
        m, n = A_np.shape
        R = np.triu(A[:n].double().cpu().numpy())
        F, _ = oracle.geqr2(A_np.astype(np.float32).astype(np.float64))
        R_or = np.triu(F[:n])
        D = oracle.row_signs(R, R_or)
        rel = np.linalg.norm(D[:, None] * R - R_or) / np.linalg.norm(R_or)
        assert rel <= 10 * n * U32, rel


def test_batched_graph_replay(q):
    mats_np = _batch(40, seed=11, m_hi=300)
    src = [_dev(a) for a in mats_np]
    work = [a.clone().t().contiguous().t() for a in src]
    plan = q.BatchedPlan(work, 0, 0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.launch(stream=s)  # warm-up outside capture (sets kernel attributes)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    eager = [w.clone() for w in work]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for w, a in zip(work, src):
            w.copy_(a)
        plan.launch(stream=torch.cuda.current_stream())
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for w, e in zip(work, eager):
        assert torch.equal(w, e)
    _check_fp64(q, plan, mats_np, work, full=False)


def test_batched_tuned_classes_up_to_512(q):
    """The full size range of the batched workload (m ~ U{32..512}) with the
    tuned size classes (the committed table: for m > 256 a multi-tile class),
    FP64 and FP32, matrix by matrix against the oracle: the classes whose
    chunks are narrower than 32 columns take the staggered staging path."""
    mats_np = _batch(40, seed=13, m_hi=512)
    assert max(a.shape[0] for a in mats_np) > 256
    outs = [_dev(a) for a in mats_np]
    plan = q.BatchedPlan(outs, 0, 0)
    nbs = plan.nb.tolist()
    assert any(nb < a.shape[0] for nb, a in zip(nbs, mats_np)), nbs  # a multi-tile class
    plan.launch()
    torch.cuda.synchronize()
    assert plan.status() == 0
    _check_fp64(q, plan, mats_np, outs, full=False)
    outs32 = [_dev(a, torch.float32) for a in mats_np]
    plan32 = q.BatchedPlan(outs32, 0, 0)
    plan32.launch()
    torch.cuda.synchronize()
    for A_np, A in zip(mats_np, outs32):
        m, n = A_np.shape
        R = np.triu(A[:n].double().cpu().numpy())
        F, _ = oracle.geqr2(A_np.astype(np.float32).astype(np.float64))
        R_or = np.triu(F[:n])
        D = oracle.row_signs(R, R_or)
        rel = np.linalg.norm(D[:, None] * R - R_or) / np.linalg.norm(R_or)
        assert rel <= 10 * n * U32, rel
