"""FP32 tile QR with the trailing-update products on the tensor cores
(qr_factor_mixed_s: TF32, or BF16x3 split products, FP32 accumulation)
against the FP64 oracle, at ragged sizes that span several tiles, flat tree
and panel domains.

Error budgets (normwise, against the oracle's FP64 Householder QR of the
same matrix). Each update product of a reduced-precision format carries the
relative error of its operands' rounding: u_p = 2^-11 for TF32 (10 fraction
bits, round to nearest) and u_p = 2^-17 for BF16x3 (x = hi + lo with 8-bit
significands leaves a 2^-18 representation error, and the dropped lo*lo
term is of the same order); FP32 storage and accumulation add u_32 = 2^-24
per operation, which grows like sqrt(n) over a factorization. So
    ||A - QR||_F / ||A||_F                 <= 10 (u_p + sqrt(n) u_32),
    ||D R - R_oracle||_F / ||R_oracle||_F  <= 10 (u_p + sqrt(n) u_32),
    ||I - Q^T Q||_F                        <= 10 n u_32,
the last independent of u_p: each reflector H = I - tau v v^T is orthogonal
whatever the accuracy of the updates that produced v, and Q is formed in
FP32. QR_PREC_F32 (the FP32 cores) is held to the same with u_p = 0. On
these inputs (kappa_F of R up to 1.3e6) the measured deviation of R follows
the backward error, about 1.2 u_p, with no growth in kappa: the budgets leave
a margin of 7x or more.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1102_5328_gb300 import inputs  # noqa: E402

U32 = 2.0 ** -24
UP = {0: 0.0, 2: 2.0 ** -11, 3: 2.0 ** -17}  # QR_PREC_F32, QR_PREC_TF32, QR_PREC_BF16X3


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1102_5328_gb300 as q
    q.lib()
    return q


CASES = [(512, 512, 64, 16, 1), (700, 300, 64, 16, 1), (333, 333, 96, 24, 1), (640, 600, 128, 32, 1),
         (1000, 1000, 128, 8, 1), (2000, 300, 64, 16, 4), (777, 250, 64, 16, 2)]


@pytest.mark.parametrize("prec", [2, 3, 1])
@pytest.mark.parametrize("m,n,nb,ib,p", CASES)
def test_mixed_factor_parity(q, prec, m, n, nb, ib, p):
    A64 = inputs.uniform_matrix(m, n, seed=m * 7 + n)
    A32 = A64.astype(np.float32)
    Ad = torch.from_numpy(np.ascontiguousarray(A32.T)).cuda().t()
    f = q.qr_factor_mixed(Ad, prec, nb, ib, p)
    Qd = q.form_q(f)
    torch.cuda.synchronize()
    assert f.status() == 0
    Q = Qd.cpu().numpy().astype(np.float64)
    R = np.triu(f.A[:n].cpu().numpy().astype(np.float64))
    Af = A32.astype(np.float64)
    F, _ = oracle.geqr2(Af)
    R_or = np.triu(F[:n])
    kF = np.linalg.norm(R_or) * np.linalg.norm(np.linalg.inv(R_or))
    res = oracle.fact_residual(Af, Q, R)
    orth = oracle.orth_residual(Q)
    D = oracle.row_signs(R, R_or)
    rel = np.linalg.norm(D[:, None] * R - R_or) / np.linalg.norm(R_or)
    b = 10 * (UP[0 if prec == 1 else prec] + math.sqrt(n) * U32)
    bo = 10 * n * U32
    print("prec %d %dx%d nb %d ib %d p %d: residual %.3e (%.2f of budget), orth %.3e (%.2f), |R| %.3e (%.2f), "
          "kappa_F %.1f" % (prec, m, n, nb, ib, p, res, res / b, orth, orth / bo, rel, rel / b, kF))
    assert res <= b and orth <= bo and rel <= b, (res, orth, rel, b, bo)


def test_tensor_core_path_differs_from_fp32_cores(q):
    """The TF32 and BF16x3 factorizations are not the FP32-core one (the
    tensor-core path ran), and BF16x3 is closer to it than TF32."""
    m = n = 512
    A32 = inputs.uniform_matrix(m, n, seed=3).astype(np.float32)
    out = {}
    for prec in (1, 2, 3):
        Ad = torch.from_numpy(np.ascontiguousarray(A32.T)).cuda().t()
        f = q.qr_factor_mixed(Ad, prec, 64, 16, 1)
        torch.cuda.synchronize()
        out[prec] = np.triu(f.A[:n].cpu().numpy().astype(np.float64))
    d_tf32 = np.linalg.norm(out[2] - out[1]) / np.linalg.norm(out[1])
    d_bf = np.linalg.norm(out[3] - out[1]) / np.linalg.norm(out[1])
    print("R distance to the FP32-core factorization: TF32 %.3e, BF16x3 %.3e" % (d_tf32, d_bf))
    assert d_tf32 > 0 and d_bf > 0 and d_bf < d_tf32
