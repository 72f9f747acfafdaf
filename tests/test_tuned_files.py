"""The committed tuning results against the committed measurements they were
derived from (CPU only): the decision tables follow from their own logs by
the oracle's restatement of the rules, and the reliability figures follow
from the logs and the exhaustive search."""
import json
import os

import pytest

from oracle import tuning

HERE = os.path.dirname(os.path.abspath(__file__))
TUNED = os.path.join(HERE, "..", "paper_1102_5328_gb300", "tuned")
SMS = 152  # the GB300 the logs were taken on


def _log(name):
    with open(os.path.join(TUNED, name)) as f:
        return [json.loads(line) for line in f if line.strip()]


def _table(name):
    with open(os.path.join(TUNED, name)) as f:
        return json.load(f)


def _flops(m, n):
    return 2.0 * m * n * n - 2.0 * n ** 3 / 3.0


def _replay_squares(log, tol):
    """Step 1 -> Property 5.1 (widened by tol) -> hull -> Heuristic 2, then
    PSPAYG over the square orders on the logged Step-2 timings."""
    perf1 = {(e["nb"], e["ib"]): 2.0 * SMS * 4.0 * e["nb"] ** 3 / e["seconds"] / 1e9 for e in log if e["kind"] == 1}
    pre = tuning.widen_ib(perf1, tuning.preselect(perf1, heuristic=2), tol)
    sec = {(e["m"], e["nb"], e["ib"]): e["seconds"] for e in log if e["kind"] == 2 and e["m"] == e["n"]}
    orders = sorted({k[0] for k in sec})
    want, count = tuning.step2_payg(orders, pre, lambda n, pr: _flops(n, n) / sec[(n,) + pr])
    return pre, want, count


@pytest.mark.parametrize("log,table,tol", [("gb300_fp64_h2.jsonl", "gb300_fp64_h2.json", 0.0),
                                           ("gb300_fp64_plain.jsonl", "gb300_fp64_plain.json", 0.02)])
def test_plain_tables_follow_from_their_logs(log, table, tol):
    L, tab = _log(log), _table(table)
    pre, want, count = _replay_squares(L, tol)
    assert tab.get("ib_tol_permille", 0) == round(1000 * tol)  # tables written before the option have none
    got = {e["m"]: (e["nb"], e["ib"]) for e in tab["entries"] if e["m"] == e["n"]}
    assert got == {n: v[0] for n, v in want.items()}
    assert count == sum(1 for e in L if e["kind"] == 2 and e["m"] == e["n"])


def test_installed_table_decides_as_the_plain_search():
    """The model-guided search (installed table) timed fewer pairs but chose
    the same (NB, IB, p) at every shape as the search without the model."""
    a, b = _table("gb300_fp64.json"), _table("gb300_fp64_plain.json")
    key = lambda t: {(e["m"], e["n"]): (e["nb"], e["ib"], e["p"]) for e in t["entries"]}
    assert key(a) == key(b)
    assert a["use_model"] == 1 and a["ib_tol_permille"] == 20 and "model" in a
    assert a["factorizations_timed"] < b["factorizations_timed"]


@pytest.mark.parametrize("rel,log,table,run", [
    ("gb300_fp64_reliability.json", "gb300_fp64_pspayg.jsonl", "gb300_fp64.json", "gb300_fp64_pspayg_run.json"),
    ("gb300_fp64_h2_reliability.json", "gb300_fp64_h2.jsonl", "gb300_fp64_h2.json", "gb300_fp64_h2_run.json")])
def test_reliability_reproduces(tmp_path, rel, log, table, run):
    from paper_1102_5328_gb300 import tune_eval
    out = str(tmp_path / "rel.json")
    j = lambda n: os.path.join(TUNED, n)
    assert tune_eval.main(["--es", j("gb300_fp64_es.jsonl"), "--es-held", j("gb300_fp64_es_held.jsonl"),
                           "--pspayg", j(log), "--table", j(table), "--tune-json", j(run),
                           "--es-json", j("gb300_fp64_es_run.json"), "--out", out]) == 0
    got, want = json.load(open(out)), _table(rel)
    for k in ("autotuned_over_grid_best", "autotuned_over_grid_best_min", "optimum_found", "tuning_seconds",
              "full_grid_seconds", "tuning_seconds_tuned_orders", "factorizations_timed_tuned_orders"):
        assert got[k] == pytest.approx(want[k], rel=1e-12), k
    # every ratio is a grid point's time over the grid best's, from the exhaustive logs
    assert all(0 < r["ratio"] <= 1 for r in got["per_shape"])


def test_committed_tables_load_and_answer_their_entries():
    """Every committed table is read by the library's own readers, and a
    lookup at each tuned shape returns that shape's entry."""
    import ctypes

    from paper_1102_5328_gb300 import _lib
    L = _lib.load()
    j = lambda n: os.path.join(TUNED, n)
    try:
        for name, prec in (("gb300_fp64.json", 0), ("gb300_fp32.json", 1)):
            L.qr_clear_tables()
            assert L.qr_load_table(j(name).encode()) == 0, name
            nb, ib, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            for e in _table(name)["entries"]:
                assert L.qr_lookup_p(e["m"], e["n"], prec, ctypes.byref(nb), ctypes.byref(ib), ctypes.byref(p)) == 0
                assert (nb.value, ib.value, p.value) == (e["nb"], e["ib"], e.get("p", 1)), (name, e)
        for name, load, look in (("gb300_chol_fp64.json", L.chol_load_table, L.chol_lookup),
                                 ("gb300_lu_fp64.json", L.lu_load_table, L.lu_lookup)):
            assert load(j(name).encode()) == 0, name
            v = ctypes.c_int()
            for e in _table(name)["entries"]:
                assert look(e["n"], ctypes.byref(v)) == 0 and v.value == e["nb"], (name, e)
    finally:
        L.qr_clear_tables()
        for name in ("gb300_fp64.json", "gb300_fp32.json"):
            L.qr_load_table(j(name).encode())


def test_write_table_round_trips(tmp_path):
    """tune.write_table writes the one-entry-per-line layout the C reader
    takes (the merged SM-budget tables go through it)."""
    import ctypes

    from paper_1102_5328_gb300 import _lib
    torch = pytest.importorskip("torch")  # tune imports torch
    from paper_1102_5328_gb300 import tune
    L = _lib.load()
    tab = {"prec": "fp64", "heuristic": 2, "entries": [
        {"m": 1000, "n": 1000, "nb": 64, "ib": 16, "p": 1, "gflops": 68.1, "sms": 0},
        {"m": 20000, "n": 500, "nb": 64, "ib": 16, "p": 32, "gflops": 311.3, "sms": 0},
        {"m": 1000, "n": 1000, "nb": 128, "ib": 8, "p": 1, "gflops": 50.0, "sms": 19}]}
    path = str(tmp_path / "w.json")
    tune.write_table(path, tab)
    assert json.load(open(path)) == tab
    try:
        L.qr_clear_tables()
        assert L.qr_load_table(path.encode()) == 0
        nb, ib, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        assert L.qr_lookup_sms(1000, 1000, 0, 19, ctypes.byref(nb), ctypes.byref(ib), ctypes.byref(p)) == 0
        assert (nb.value, ib.value, p.value) == (128, 8, 1)
        assert L.qr_lookup_p(22000, 480, 0, ctypes.byref(nb), ctypes.byref(ib), ctypes.byref(p)) == 0
        assert (nb.value, ib.value, p.value) == (64, 16, 32)
    finally:
        L.qr_clear_tables()
        for name in ("gb300_fp64.json", "gb300_fp32.json"):
            L.qr_load_table(os.path.join(TUNED, name).encode())


def test_tune_eval_widening_is_the_oracles():
    """tune_eval's replay of the IB tolerance applies the oracle's rule
    (random Step-1 tables, several tolerances)."""
    import random

    from paper_1102_5328_gb300 import tune_eval
    rng = random.Random(5)
    for _ in range(50):
        perf = {(nb, ib): rng.uniform(100, 200) for nb in (64, 96, 128) for ib in (8, 16, 32)}
        pre = tuning.preselect(perf, heuristic=2)
        for tol in (0.0, 0.01, 0.05, 0.2):
            assert tune_eval.widen(perf, pre, tol) == tuning.widen_ib(perf, pre, tol)


def test_ib_tolerance_sweep_reproduces():
    from paper_1102_5328_gb300 import tune_eval
    import io
    import contextlib
    j = lambda n: os.path.join(TUNED, n)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert tune_eval.main(["--es", j("gb300_fp64_es.jsonl"), "--es-held", j("gb300_fp64_es_held.jsonl"),
                               "--pspayg", j("gb300_fp64_h2.jsonl"), "--table", j("gb300_fp64_h2.json"),
                               "--ib-tols", "0,5,10,15,20,30,50,100"]) == 0
    got = json.loads(buf.getvalue())["replayed_ib_tolerance_permille"]
    want = _table("gb300_fp64_ib_tol_sweep.json")["replayed_ib_tolerance_permille"]
    assert got.keys() == want.keys()
    for k in want:
        for f in ("preselected", "step2_seconds_6runs", "mean_ratio", "min_ratio"):
            assert got[k][f] == pytest.approx(want[k][f], rel=1e-12), (k, f)
    # tolerance 0 is the paper's Heuristic 2
    assert want["0"]["mean_ratio"] == pytest.approx(_table("gb300_fp64_h2_reliability.json")["replayed_heuristics"]["H2"]["mean_ratio"])


def test_installed_table_replays_as_a_model_guided_search():
    """The installed table's own log (Step 1, every Step-2 timing, the
    model's logged predictions, kind 4) replayed by the rules: Step 1 ->
    Heuristic 2 widened by the 2 % IB tolerance; at each shape, ascending
    n, the pairs timed are the model's k = 1 best, extended down its ranking
    while the last one timed was the fastest so far, and all survivors when
    a timed pair's measured / predicted ratio differs from the top-ranked
    one's by more than e^0.25; shapes without predictions are timed in full;
    prune-as-you-go between square orders. The logged timings are exactly
    those pairs and the table holds each shape's fastest."""
    import math
    L, tab = _log("gb300_fp64_pspayg.jsonl"), _table("gb300_fp64.json")
    perf1 = {(e["nb"], e["ib"]): 2.0 * SMS * 4.0 * e["nb"] ** 3 / e["seconds"] / 1e9 for e in L if e["kind"] == 1}
    surv = tuning.widen_ib(perf1, tuning.preselect(perf1, heuristic=2), 0.02)
    sec2 = {(e["m"], e["n"], e["nb"], e["ib"]): e["seconds"] for e in L if e["kind"] == 2}
    pred = {(e["m"], e["n"], e["nb"], e["ib"]): e["seconds"] for e in L if e["kind"] == 4}
    shapes = sorted({(e["m"], e["n"]) for e in L if e["kind"] == 2}, key=lambda s: (s[1], s[0]))
    k, guided = 1, 0
    timed_log = {}
    for e in L:
        if e["kind"] == 2:
            timed_log.setdefault((e["m"], e["n"]), set()).add((e["nb"], e["ib"]))
    entries = {(e["m"], e["n"]): (e["nb"], e["ib"]) for e in tab["entries"]}
    for m, n in shapes:
        if any((m, n) + pr in pred for pr in surv):
            guided += 1
            rank = sorted(range(len(surv)), key=lambda c: pred[(m, n) + surv[c]])
            timed = [rank[0]]
            r = 1
            while r < len(surv) and min(timed, key=lambda c: (sec2[(m, n) + surv[c]], timed.index(c))) == timed[-1]:
                timed.append(rank[r])
                r += 1
            scale = math.log(sec2[(m, n) + surv[timed[0]]]) - math.log(pred[(m, n) + surv[timed[0]]])
            if any(abs(math.log(sec2[(m, n) + surv[c]]) - math.log(pred[(m, n) + surv[c]]) - scale) > 0.25
                   for c in timed[1:]):
                timed += rank[r:]
        else:
            timed = list(range(len(surv)))
        pairs = [surv[c] for c in timed]
        assert set(pairs) == timed_log[(m, n)], (m, n)
        perf = {pr: _flops(m, n) / sec2[(m, n) + pr] for pr in pairs}
        assert entries[(m, n)] == max(pairs, key=lambda pr: (perf[pr], -pr[0])), (m, n)
        if m == n:
            keep = tuning.payg_prune(pairs, perf)
            surv = [pr for pr in surv if pr not in pairs or pr in keep]
    assert guided >= 3  # the third square order on
