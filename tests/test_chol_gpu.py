"""Tile Cholesky on the GPU (chol_factor_d through the C ABI) against the
oracle's column Cholesky, at sizes that span several tiles with ragged
edges; non-SPD detection; determinism; the bench-size factorization through
sampled entries of L L^T; and the NB tuner replayed through the oracle's
restatement of the paper's rules.

Budgets: Cholesky is backward stable with ||A - L L^T|| <= c n u ||A||; on
these inputs (G G^T / n + I, eigenvalues in about [1, 5]) the factor is
well conditioned, so L agrees with the oracle's to the same order:
||A - L L^T||_F / ||A||_F <= 10 n u and ||L - L_oracle||_F / ||L_oracle||_F
<= 10 n u, u = 2^-53."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import tuning  # noqa: E402
from paper_1102_5328_gb300 import inputs  # noqa: E402

U = 2.0 ** -53


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1102_5328_gb300 as q
    q.lib()
    return q


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()


@pytest.mark.parametrize("n,nb", [(64, 64), (100, 32), (333, 96), (777, 64), (1000, 128), (512, 256), (513, 256),
                                  (40, 16)])
def test_chol_parity(q, n, nb):
    A = inputs.spd_matrix(n, seed=n + nb)
    Ad = _dev(A)
    f = q.chol_factor(Ad, nb)
    torch.cuda.synchronize()
    assert f.status() == (0, -1)
    out = Ad.cpu().numpy()
    L = np.tril(out)
    assert np.array_equal(np.triu(out, 1), np.triu(A, 1))  # upper triangle untouched
    Lo, info = oracle.potrf(A)
    assert info == 0
    res = oracle.chol_residual(A, L)
    rel = np.linalg.norm(L - Lo) / np.linalg.norm(Lo)
    assert res <= 10 * n * U and rel <= 10 * n * U, (res, rel)


def test_chol_not_positive_definite(q):
    """A pivot that is not positive (column 150, in the third tile row of 64)
    sets QR_DEV_NOT_SPD and reports that column, as the oracle's info does."""
    n, nb, bad = 300, 64, 150
    A = inputs.spd_matrix(n, seed=8)
    A[bad, bad] -= 1e3
    _, info = oracle.potrf(A)
    assert info == bad + 1
    f = q.chol_factor(_dev(A), nb)
    st, col = f.status()
    assert st & q.QR_DEV_NOT_SPD and col == bad


def test_chol_deterministic_and_order_free(q):
    """Every tile sees its operations in a fixed order, so the result does
    not depend on the schedule: bitwise equal to a run with one worker."""
    n, nb = 700, 64
    A = inputs.spd_matrix(n, seed=9)
    f1 = q.chol_factor(_dev(A), nb)
    q.qr_set_option(q.QR_OPT_GRID_LIMIT, 1)
    try:
        f2 = q.chol_factor(_dev(A), nb)
        torch.cuda.synchronize()
    finally:
        q.qr_set_option(q.QR_OPT_GRID_LIMIT, 0)
    assert torch.equal(torch.tril(f1.A), torch.tril(f2.A))


@pytest.mark.slow
def test_chol_bench_size_sampled(q):
    """N = 10000 (the benchmark's size, nb from the table): sampled entries of
    L L^T equal A's within 10 n u ||a_i|| ||a_j||-style bounds
    (|(L L^T - A)_ij| <= 10 n u ||L_i|| ||L_j||), and the diagonal of L is
    positive."""
    n = 10000
    A = inputs.spd_matrix(n, seed=10000)
    Ad = _dev(A)
    f = q.chol_factor(Ad)
    torch.cuda.synchronize()
    assert f.status()[0] == 0
    rng = np.random.default_rng(3)
    rows = rng.integers(0, n, size=40)
    Lrows = {int(i): Ad[int(i), : int(i) + 1].cpu().numpy() for i in rows}
    for i in rows:
        for j in rows:
            i_, j_ = int(max(i, j)), int(min(i, j))
            li, lj = Lrows[i_], Lrows[j_]
            k = j_ + 1
            lhs = float(li[:k] @ lj[:k])
            assert abs(lhs - A[i_, j_]) <= 10 * n * U * np.linalg.norm(li) * np.linalg.norm(lj), (i_, j_)
    assert np.all(np.diag(Ad.cpu().numpy()) > 0)


def test_chol_tuner_matches_oracle_replay(q, tmp_path):
    table, log = str(tmp_path / "ct.json"), str(tmp_path / "cl.jsonl")
    res = q.chol_tune([256, 512, 768], heuristic=2, reps=2, table=table, log=log)
    with open(log) as f:
        entries = [json.loads(line) for line in f if line.strip()]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    perf1 = {(e["nb"], 1): 2.0 * sms * 2.0 * e["nb"] ** 3 / e["seconds"] / 1e9 for e in entries if e["kind"] == 11}
    assert sorted(perf1) == [(nb, 1) for nb in range(32, 257, 32)]
    pre = tuning.preselect(perf1, heuristic=2)
    step2 = {(e["n"], e["nb"]): e["n"] ** 3 / 3.0 / e["seconds"] for e in entries if e["kind"] == 12}
    want, count = tuning.step2_payg([256, 512, 768], pre, lambda n, pr: step2[(n, pr[0])])
    assert count == len(step2) == res["factorizations_timed"]
    tab = json.load(open(table))
    assert {e["n"]: e["nb"] for e in tab["entries"]} == {n: v[0][0] for n, v in want.items()}
    import ctypes
    out = ctypes.c_int()
    assert q.lib().chol_lookup(600, ctypes.byref(out)) == 0 and out.value == want[512][0][0]
    # leave no tuned table behind for later tests
    path = os.path.join(q._TUNED_DIR, "gb300_chol_fp64.json")
    if os.path.exists(path):
        q.lib().chol_load_table(path.encode())
