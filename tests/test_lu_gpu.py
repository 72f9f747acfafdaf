"""Tile LU with incremental pivoting on the GPU (lu_factor_d through the C
ABI) against the oracle's task-by-task restatement (oracle/lu.py) at sizes
that span several tiles with ragged edges; zero-pivot detection;
determinism; and, at the benchmark's order, the GPU's factors checked by the
oracle applying them to a right-hand side.

Budgets: both sides make the same pivot decisions (identical records) and
differ only by rounding (the GPU's updates are fused multiply-adds), so the
factors agree to 1e-10 of max |U|; the oracle's transformations built from
the GPU's factors take A to the GPU's U within 50 n u max |A|; a solve with
the GPU's factors has backward error ||A x - b|| / (||A|| ||x||) <= 100 n u.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import lu  # noqa: E402
from paper_1102_5328_gb300 import inputs  # noqa: E402

U = 2.0 ** -53


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1102_5328_gb300 as q
    q.lib()
    yield q
    q.qr_set_option(q.QR_OPT_GRID_LIMIT, 0)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x.T)).cuda().t()


def _piv_equal(pg, po, n, nb):
    NT = (n + nb - 1) // nb
    pg = pg.reshape(NT, NT, nb)  # [k][i][c]
    for k in range(NT):
        nk = min(nb, n - k * nb)
        for i in range(k, NT):
            if not np.array_equal(pg[k, i, :nk], po[i, k, :nk]):
                return (i, k)
    return None


@pytest.mark.parametrize("n,nb", [(64, 64), (100, 32), (333, 48), (500, 64), (777, 64), (40, 8), (129, 16),
                                  (256, 64)])
def test_lu_parity(q, n, nb):
    A = inputs.uniform_matrix(n, n, seed=n + nb)
    Ad = _dev(A)
    f = q.lu_factor(Ad, nb)
    torch.cuda.synchronize()
    assert f.status() == (0, -1)
    Fg = Ad.cpu().numpy()
    pg = f.piv.cpu().numpy().astype(np.int64)
    Fo, po, info = lu.getrf_incpiv(A, nb)
    assert info == 0
    assert _piv_equal(pg, po, n, nb) is None
    scale = np.abs(np.triu(Fo)).max()
    assert np.abs(Fg - Fo).max() <= 1e-10 * max(1.0, scale), np.abs(Fg - Fo).max()
    # the GPU's factors, applied by the oracle, take A to the GPU's U
    NT = (n + nb - 1) // nb
    pr = np.transpose(pg.reshape(NT, NT, nb), (1, 0, 2))  # [i][k][c]
    Y = lu.apply_incpiv(Fg, pr, nb, A)
    assert np.abs(np.triu(Y) - np.triu(Fg)).max() <= 50 * n * U * np.abs(A).max() * max(1.0, scale)
    assert np.abs(np.tril(Y, -1)).max() <= 50 * n * U * np.abs(A).max() * max(1.0, scale)


def test_lu_zero_pivot_reported(q):
    """A zero column (column 150, in the third tile column of 64) makes that
    column's pivot zero: QR_DEV_SINGULAR and the column, as the oracle's
    info says."""
    n, nb, bad = 300, 64, 150
    A = inputs.uniform_matrix(n, n, seed=8)
    A[:, bad] = 0.0
    _, _, info = lu.getrf_incpiv(A, nb)
    assert info == bad + 1
    f = q.lu_factor(_dev(A), nb)
    st, col = f.status()
    assert st & q.QR_DEV_SINGULAR and col == bad


def test_lu_deterministic_and_order_free(q):
    """Every tile sees its operations in a fixed order: the result does not
    depend on the schedule (bitwise equal to a run with one worker)."""
    n, nb = 700, 64
    A = inputs.uniform_matrix(n, n, seed=9)
    f1 = q.lu_factor(_dev(A), nb)
    q.qr_set_option(q.QR_OPT_GRID_LIMIT, 1)
    try:
        f2 = q.lu_factor(_dev(A), nb)
        torch.cuda.synchronize()
    finally:
        q.qr_set_option(q.QR_OPT_GRID_LIMIT, 0)
    assert torch.equal(f1.A, f2.A) and torch.equal(f1.piv, f2.piv)


@pytest.mark.slow
def test_lu_bench_size_solve(q):
    """N = 10000, NB = 64 (the benchmark's configuration): a right-hand side
    solved with the GPU's factors by the oracle's transformations and back
    substitution has backward error <= 100 n u."""
    n, nb = 10000, 64
    A = inputs.uniform_matrix(n, n, seed=n)
    Ad = _dev(A)
    f = q.lu_factor(Ad, nb)
    torch.cuda.synchronize()
    assert f.status()[0] == 0
    Fg = Ad.cpu().numpy()
    NT = (n + nb - 1) // nb
    pr = np.transpose(f.piv.cpu().numpy().astype(np.int64).reshape(NT, NT, nb), (1, 0, 2))
    b = np.random.default_rng(1).standard_normal((n, 1))
    x = lu.lu_solve(Fg, pr, nb, b)
    r = A @ x - b
    assert np.linalg.norm(r) / (np.linalg.norm(A, 2) * np.linalg.norm(x)) <= 100 * n * U


def test_lu_tuner_matches_oracle_replay(q, tmp_path):
    """lu_tune (Step 1 over NB 16..64, Heuristic 2, Step 2 with
    prune-as-you-go) replayed by the oracle's restatement of the rules from
    its own log."""
    import ctypes
    import json
    import os

    from oracle import tuning
    table, log = str(tmp_path / "lt.json"), str(tmp_path / "ll.jsonl")
    try:
        res = q.lu_tune([256, 512, 768], heuristic=2, reps=2, table=table, log=log)
        with open(log) as f:
            entries = [json.loads(line) for line in f if line.strip()]
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        perf1 = {(e["nb"], 1): 2.0 * sms * 2.0 * e["nb"] ** 3 / e["seconds"] / 1e9 for e in entries if e["kind"] == 21}
        assert sorted(perf1) == [(nb, 1) for nb in range(16, 65, 8)]
        pre = tuning.preselect(perf1, heuristic=2)
        step2 = {(e["n"], e["nb"]): 2.0 * e["n"] ** 3 / 3.0 / e["seconds"] for e in entries if e["kind"] == 22}
        want, count = tuning.step2_payg([256, 512, 768], pre, lambda n, pr: step2[(n, pr[0])])
        assert count == len(step2) == res["factorizations_timed"]
        tab = json.load(open(table))
        assert {e["n"]: e["nb"] for e in tab["entries"]} == {n: v[0][0] for n, v in want.items()}
        out = ctypes.c_int()
        assert q.lib().lu_lookup(600, ctypes.byref(out)) == 0 and out.value == want[512][0][0]
    finally:
        q.lib().lu_clear_table()
        path = os.path.join(q._TUNED_DIR, "gb300_lu_fp64.json")
        if os.path.exists(path):
            q.lib().lu_load_table(path.encode())
