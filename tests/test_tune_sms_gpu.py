"""The SM-count axis of the tuner (the GPU counterpart of the paper's core
counts, Sec. 6.1): QR_OPT_SM_BUDGET caps the persistent factorization's
workers, qr_tune records the budget of every Step-2 timing and table entry,
and qr_lookup_sms serves a (shape, budget) request from the closest tuned
budget, then the closest tuned shape."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import tuning  # noqa: E402
from paper_1102_5328_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1102_5328_gb300 as q
    q.lib()
    yield q
    q.qr_set_option(q.QR_OPT_SM_BUDGET, 0)
    q.lib().qr_clear_tables()
    for name in ("gb300_fp64.json", "gb300_fp32.json"):
        path = os.path.join(q._TUNED_DIR, name)
        if os.path.exists(path):
            q.lib().qr_load_table(path.encode())


def _factor(q, A_np, nb, ib, budget, trace=False):
    q.qr_set_option(q.QR_OPT_SM_BUDGET, budget)
    try:
        A = torch.from_numpy(np.ascontiguousarray(A_np.T)).cuda().t()
        # T's storage has entries the factorization never writes (below the
        # diagonal of each IB x IB block, tiles above the diagonal): start
        # every run from zeros so the comparison sees only what was computed
        t_elems, _ = q.qr_workspace(A.shape[0], A.shape[1], nb, ib, A.dtype)
        T = torch.zeros(max(t_elems, 1), dtype=A.dtype, device="cuda")
        buf = None
        if trace:
            ntasks = q.qr_task_count(A.shape[0], A.shape[1], nb, ib)
            buf = torch.full((ntasks, 4), -1, dtype=torch.int64, device="cuda")
            q.qr_set_trace(buf)
        try:
            f = q.qr_factor(A, nb, ib, T=T)
            torch.cuda.synchronize()
        finally:
            if trace:
                q.qr_set_trace(None)
        assert f.status() == 0
        return f, buf
    finally:
        q.qr_set_option(q.QR_OPT_SM_BUDGET, 0)


@pytest.mark.parametrize("budget", [1, 4, 19])
def test_budget_caps_the_workers(q, budget):
    """With a budget of b SMs the persistent kernel runs 2b CTAs, so its
    tasks land on at most 2b distinct SMs; the result is bitwise that of the
    whole GPU (every tile sees the same operation sequence)."""
    m = n = 640
    nb, ib = 64, 16
    A_np = inputs.uniform_matrix(m, n, seed=41)
    f_all, _ = _factor(q, A_np, nb, ib, 0)
    f_b, buf = _factor(q, A_np, nb, ib, budget, trace=True)
    _, _, sm, _, _, _ = q.read_trace(buf, q.qr_task_count(m, n, nb, ib))
    assert len(set(sm.tolist())) <= 2 * budget
    assert torch.equal(f_all.A, f_b.A) and torch.equal(f_all.T, f_b.T)


def test_tuner_per_budget_matches_oracle_replay(q, tmp_path):
    """tune.py --sm-budgets: Step 1 once (shared log), Step 2 under each
    budget; the merged table's entries per budget are the oracle's decisions
    on that budget's logged timings, and qr_lookup_sms answers from them."""
    from paper_1102_5328_gb300 import tune
    table = str(tmp_path / "sms_table.json")
    log = str(tmp_path / "sms_log.jsonl")
    shapes = "256,512,768"
    tune.main(["--mode", "pspayg", "--heuristic", "2", "--reps", "2", "--prec", "f32", "--ns", shapes,
               "--table", table, "--log", log, "--sm-budgets", "8,0"])
    with open(log) as f:
        entries = [json.loads(line) for line in f if line.strip()]
    tab = json.load(open(table))
    assert tab["sm_budgets"] == [8, 0]
    assert len([e for e in entries if e["kind"] == 1]) == len(tuning.grid_pairs())  # Step 1 once
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    perf1 = {(e["nb"], e["ib"]): 2.0 * sms * 4.0 * e["nb"] ** 3 / e["seconds"] / 1e9
             for e in entries if e["kind"] == 1}
    pre = tuning.preselect(perf1, heuristic=2)
    for budget in (8, 0):
        perf = {(e["m"], e["nb"], e["ib"]): 2.0 * e["m"] ** 3 * (2.0 / 3.0) / e["seconds"]
                for e in entries if e["kind"] == 2 and e["sms"] == budget}

        def measure(n, pr, perf=perf):
            return perf[(n, pr[0], pr[1])]

        want, count = tuning.step2_payg([256, 512, 768], pre, measure)
        assert count == len(perf)
        got = {e["m"]: (e["nb"], e["ib"]) for e in tab["entries"] if e["sms"] == budget}
        assert got == {n: v[0] for n, v in want.items()}, budget
        for n in (256, 600, 768):
            assert q.qr_lookup_sms(n, n, torch.float32, budget)[:2] == want[tuning.nearest(n, [256, 512, 768])][0]
    # a budget between the tuned ones takes the closer (ties to the smaller)
    assert q.qr_lookup_sms(512, 512, torch.float32, 9)[:2] == \
        {e["m"]: (e["nb"], e["ib"]) for e in tab["entries"] if e["sms"] == 8}[512]
