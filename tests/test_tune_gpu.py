"""The empirical tuner run on the GPU (qr_tune through the C ABI), its
decisions replayed through the oracle's restatement of the paper's rules.

qr_tune (PSPAYG, Heuristic 2) times Step 1 (the TSMQR kernel batch for all
119 (NB, IB) pairs, Sec. 5) and Step 2 (the factorization for the survivors
at each order, prune as you go, Secs. 6.1 and 6.3) on the device and logs
every measurement. From the logged numbers alone, oracle.tuning must reach
the same preselection (Property 5.1, the upper hull of Property 5.2,
Heuristic 2), the same survivors at each order (Property 6.1) and the same
decision table.
"""
import ctypes
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import tuning  # noqa: E402


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1102_5328_gb300 as q
    q.lib()
    yield q
    # qr_tune installs its table in-process: put the committed tables back
    # for the tests that follow
    for name in ("gb300_fp64.json", "gb300_fp32.json"):
        path = os.path.join(q._TUNED_DIR, name)
        if os.path.exists(path):
            q.lib().qr_load_table(path.encode())


def _flops(m, n):
    return 2.0 * m * n * n - 2.0 * n ** 3 / 3.0


def _read_log(path):
    with open(path) as f:
        return [json.loads(line) for line in f if line.strip()]


def run_tune(q, shapes, tmp_path, prec, reps=2, heuristic=2, mode=0, tag="t", ib_tol=0):
    from paper_1102_5328_gb300 import tune
    table = str(tmp_path / ("%s_table.json" % tag))
    log = str(tmp_path / ("%s_log.jsonl" % tag))
    res = tune.run(shapes, "es" if mode else "pspayg", heuristic, reps, prec, table, log, ib_tol=ib_tol)
    return res, json.load(open(table)), _read_log(log)


def replay(log, shapes, sms, heuristic=2, ib_tol=0.0):
    """The tuner's decisions recomputed by the oracle from its own log."""
    perf1 = {(e["nb"], e["ib"]): 2.0 * sms * 4.0 * e["nb"] ** 3 / e["seconds"] / 1e9
             for e in log if e["kind"] == 1}
    pre = tuning.widen_ib(perf1, tuning.preselect(perf1, heuristic=heuristic), ib_tol)
    step2 = {}
    for e in log:
        if e["kind"] == 2:
            step2[(e["m"], e["n"], e["nb"], e["ib"])] = _flops(e["m"], e["n"]) / e["seconds"] / 1e9
    surv = list(pre)
    measured, table = {}, {}
    for m, n in sorted(shapes, key=lambda s: (s[1], s[0])):
        perf_n = {pr: step2[(m, n) + pr] for pr in surv}
        measured[(m, n)] = sorted(surv)
        best = max(surv, key=lambda pr: (perf_n[pr], -pr[0]))
        table[(m, n)] = best
        if m == n:
            surv = tuning.payg_prune(surv, perf_n)
    return perf1, pre, measured, table


def test_tuner_on_gpu_matches_oracle_replay(q, tmp_path):
    shapes = [(256, 256), (512, 512), (768, 768)]
    res, tab, log = run_tune(q, shapes, tmp_path, q.QR_PREC_F64)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    perf1, pre, measured, table = replay(log, shapes, sms)
    # Step 1 covered the whole grid, once per pair
    assert sorted(perf1) == sorted(tuning.grid_pairs())
    assert len([e for e in log if e["kind"] == 1]) == len(tuning.grid_pairs())
    assert 1 <= len(pre) <= 8
    # Step 2 measured exactly the oracle's survivors at each order
    got = {}
    for e in log:
        if e["kind"] == 2:
            got.setdefault((e["m"], e["n"]), []).append((e["nb"], e["ib"]))
    assert {k: sorted(v) for k, v in got.items()} == measured
    assert measured[(256, 256)] == sorted(pre)
    assert all(e["reps"] == 2 for e in log if e["kind"] == 2)
    # the decision table is the oracle's
    entries = {(e["m"], e["n"]): (e["nb"], e["ib"]) for e in tab["entries"]}
    assert entries == table
    assert all(e["p"] == 1 for e in tab["entries"])  # squares: flat tree
    # the wall-time accounting
    assert res["factorizations_timed"] == sum(len(v) for v in measured.values())
    assert 0 < res["step1_seconds"] and 0 < res["step2_seconds"]
    assert res["step1_seconds"] + res["step2_seconds"] <= res["seconds"] * 1.001
    # the in-process table now answers qr_lookup with the tuned pairs, and
    # an untuned order takes the closest tuned one (Sec. 6.1)
    for (m, n), pr in table.items():
        assert q.qr_lookup(m, n) == pr
    assert q.qr_lookup(400, 400) == table[(512, 512)]
    assert q.qr_lookup(300, 300) == table[(256, 256)]


def test_tuner_resumes_from_its_log(q, tmp_path):
    """A second run over the same log measures nothing again and reaches the
    same table (measurements already logged are reused)."""
    shapes = [(256, 256), (384, 384)]
    res1, tab1, log1 = run_tune(q, shapes, tmp_path, q.QR_PREC_F32, tag="r")
    res2, tab2, log2 = run_tune(q, shapes, tmp_path, q.QR_PREC_F32, tag="r")
    assert res2["factorizations_timed"] == 0 and res2["step1_seconds"] == 0
    assert len(log2) == len(log1)
    assert tab1["entries"] == tab2["entries"]


def test_tuner_ib_tolerance_replays(q, tmp_path):
    """QR_OPT_TUNE_IB_TOL (here 5 %): each preselected NB also brings the IBs
    within 5 % of its best IB's Step-1 rate; Step 2 measures exactly the
    oracle's widened survivors and the table is the oracle's decision."""
    shapes = [(256, 256), (512, 512), (768, 768)]
    res, tab, log = run_tune(q, shapes, tmp_path, q.QR_PREC_F64, tag="w", ib_tol=50)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    perf1, pre, measured, table = replay(log, shapes, sms, ib_tol=0.05)
    plain = tuning.preselect(perf1, heuristic=2)
    assert set(plain) <= set(pre)
    got = {}
    for e in log:
        if e["kind"] == 2:
            got.setdefault((e["m"], e["n"]), []).append((e["nb"], e["ib"]))
    assert {k: sorted(v) for k, v in got.items()} == measured
    assert measured[(256, 256)] == sorted(pre)
    entries = {(e["m"], e["n"]): (e["nb"], e["ib"]) for e in tab["entries"]}
    assert entries == table
    assert tab["ib_tol_permille"] == 50 and q.qr_get_option(q.QR_OPT_TUNE_IB_TOL) == 0
