"""The learned cost model inside the empirical search (qr_tune with
use_model = k), and the MultCallFlushLRU variant of Step 1, on the GPU.

The model-guided Step 2 is replayed from the tuner's own log: at every
square order from the third on where the model ranked the survivors (logged
predictions, kind 4), the pairs timed must be exactly the k predicted
fastest, extended down the ranking while the last one timed was the fastest
so far, and all of them when a timed pair's measured / predicted ratio
differed from the top-ranked pair's by more than e^0.25. The decision
table must be the best timed pair; survivors left untimed are not pruned
(Property 6.1 needs a measurement). The saved model is evaluated by the
oracle's fp64 forward pass: it fits the timings it was trained on, and
qr_model_propose returns its least-predicted pair.
"""
import ctypes
import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlp, tuning  # noqa: E402

TRUST = 0.25


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1102_5328_gb300 as q
    q.lib()
    yield q
    for name in ("gb300_fp64.json", "gb300_fp32.json"):
        path = os.path.join(q._TUNED_DIR, name)
        if os.path.exists(path):
            q.lib().qr_load_table(path.encode())
        else:
            q.lib().qr_clear_tables()


def _flops(m, n):
    return 2.0 * m * n * n - 2.0 * n ** 3 / 3.0


def _run(q, shapes, tmp_path, prec, tag, use_model=0, flush=False, reps=2):
    from paper_1102_5328_gb300 import tune
    table = str(tmp_path / ("%s_table.json" % tag))
    log = str(tmp_path / ("%s_log.jsonl" % tag))
    res = tune.run(shapes, "pspayg", 2, reps, prec, table, log, use_model=use_model, flush=flush)
    with open(log) as f:
        entries = [json.loads(line) for line in f if line.strip()]
    return res, json.load(open(table)), entries


def _replay_guided(log, shapes, sms, k, step1_kind=1):
    perf1 = {(e["nb"], e["ib"]): 2.0 * sms * 4.0 * e["nb"] ** 3 / e["seconds"] / 1e9
             for e in log if e["kind"] == step1_kind}
    pre = tuning.preselect(perf1, heuristic=2)
    sec2 = {(e["m"], e["n"], e["nb"], e["ib"]): e["seconds"] for e in log if e["kind"] == 2}
    pred = {(e["m"], e["n"], e["nb"], e["ib"]): e["seconds"] for e in log if e["kind"] == 4}
    surv = list(pre)
    out, guided_orders = {}, 0
    for idx, (m, n) in enumerate(sorted(shapes, key=lambda s: (s[1], s[0]))):
        if any((m, n) + pr in pred for pr in surv):
            guided_orders += 1
            assert idx >= 2 and len(surv) > k
            assert all((m, n) + pr in pred for pr in surv)
            rank = sorted(range(len(surv)), key=lambda c: pred[(m, n) + surv[c]])  # stable, like the tuner
            timed = [rank[r] for r in range(k)]
            r = k

            def fastest():
                return min(timed, key=lambda c: (sec2[(m, n) + surv[c]], timed.index(c)))

            while r < len(surv) and fastest() == timed[-1]:
                timed.append(rank[r])
                r += 1
            scale = math.log(sec2[(m, n) + surv[timed[0]]]) - math.log(pred[(m, n) + surv[timed[0]]])
            if any(abs(math.log(sec2[(m, n) + surv[c]]) - math.log(pred[(m, n) + surv[c]]) - scale) > TRUST
                   for c in timed[1:]):
                timed += rank[r:]
        else:
            timed = list(range(len(surv)))
        pairs = [surv[c] for c in timed]
        perf = {pr: _flops(m, n) / sec2[(m, n) + pr] / 1e9 for pr in pairs}
        best = max(pairs, key=lambda pr: (perf[pr], -pr[0]))
        out[(m, n)] = (sorted(pairs), best)
        if m == n:
            keep = tuning.payg_prune(pairs, perf)
            surv = [pr for pr in surv if pr not in pairs or pr in keep]
    return pre, out, guided_orders


def _model_params(tab):
    md = tab["model"]
    p = np.array(md["params"], dtype=np.float64)
    params = [p[0:256].reshape(64, 4), p[256:320], p[320:4416].reshape(64, 64), p[4416:4480],
              p[4480:4544].reshape(1, 64), p[4544:4545]]
    return md, params


def _predict(md, params, m, n, pairs):
    X = np.stack([mlp.features(m, n, nb, ib) for nb, ib in pairs])
    Z = (X - np.array(md["mean"])) / np.array(md["sd"])
    y, _ = mlp.forward(params, Z)
    return np.exp(y + md["ymean"])


def test_model_guided_search_replays(q, tmp_path):
    shapes = [(n, n) for n in (256, 384, 512, 640, 768, 1024, 1280)]
    k = 1
    res, tab, log = _run(q, shapes, tmp_path, q.QR_PREC_F64, "g", use_model=k)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    pre, out, guided = _replay_guided(log, shapes, sms, k)
    got = {}
    for e in log:
        if e["kind"] == 2:
            got.setdefault((e["m"], e["n"]), []).append((e["nb"], e["ib"]))
    assert {s: sorted(v) for s, v in got.items()} == {s: v[0] for s, v in out.items()}
    entries = {(e["m"], e["n"]): (e["nb"], e["ib"]) for e in tab["entries"]}
    assert entries == {s: v[1] for s, v in out.items()}
    assert tab["use_model"] == k and res["model_seconds"] > 0
    assert res["model_fallbacks"] <= guided
    # the saved model: trained on every Step-2 timing, it fits them
    md, params = _model_params(tab)
    assert sorted(tuple(p) for p in md["pairs"]) == sorted(pre)
    timed = [(e["m"], e["n"], e["nb"], e["ib"], e["seconds"]) for e in log if e["kind"] == 2]
    err = [math.log(_predict(md, params, m, n, [(nb, ib)])[0] / s) for m, n, nb, ib, s in timed]
    assert np.sqrt(np.mean(np.square(err))) < 0.15, err
    # qr_model_propose: the least-predicted pair of the saved model, after a
    # reload of the table from disk
    L = q.lib()
    L.qr_clear_tables()
    assert L.qr_load_table(str(tmp_path / "g_table.json").encode()) == 0
    work = torch.empty(4 << 20, dtype=torch.uint8, device="cuda")
    nb, ib, sec = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    for m, n in [(900, 900), (2000, 2000), (3000, 1000)]:
        rc = L.qr_model_propose(m, n, q.QR_PREC_F64, ctypes.byref(nb), ctypes.byref(ib), ctypes.byref(sec),
                                ctypes.c_void_p(work.data_ptr()), work.numel(), q._stream_ptr())
        assert rc == 0
        pairs = [tuple(p) for p in md["pairs"]]
        pr = _predict(md, params, m, n, pairs)
        assert (nb.value, ib.value) in pairs
        # FP32 on the GPU vs fp64 here: the proposal is (one of) the least predicted
        assert pr[pairs.index((nb.value, ib.value))] <= pr.min() * (1 + 1e-4)
        assert abs(sec.value / pr.min() - 1) < 1e-3
    # no model for a precision that was not tuned with one
    L.qr_clear_tables()
    assert L.qr_model_propose(900, 900, q.QR_PREC_F32, ctypes.byref(nb), ctypes.byref(ib), None,
                              ctypes.c_void_p(work.data_ptr()), work.numel(), q._stream_ptr()) == 1


def test_model_times_no_more_than_plain_search(q, tmp_path):
    """On the same orders the model-guided search times at most as many
    factorizations as the plain PSPAYG search (FP32, short runs)."""
    shapes = [(n, n) for n in (256, 512, 768, 1024, 1536, 2048)]
    r0, t0, _ = _run(q, shapes, tmp_path, q.QR_PREC_F32, "p0")
    r1, t1, _ = _run(q, shapes, tmp_path, q.QR_PREC_F32, "p1", use_model=1)
    assert r1["factorizations_timed"] <= r0["factorizations_timed"]


def test_step1_multcallflushlru(q, tmp_path):
    """Step 1 as MultCallFlushLRU: more workspace (operand copies covering
    two L2 capacities), a positive time per launch, and a tuner run whose
    preselection the oracle reproduces from the flushed timings (kind 5)."""
    L = q.lib()
    b0, b1 = ctypes.c_int64(), ctypes.c_int64()
    assert L.qr_step1_workspace(64, q.QR_PREC_F64, 0, ctypes.byref(b0)) == 0
    assert L.qr_step1_workspace(64, q.QR_PREC_F64, 1, ctypes.byref(b1)) == 0
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    assert b1.value >= 2 * l2 + b0.value and b1.value % b0.value == 0
    work = torch.empty(b1.value, dtype=torch.uint8, device="cuda")
    s, g = ctypes.c_double(), ctypes.c_double()
    for flush in (0, 1):
        assert L.qr_step1_time(64, 8, q.QR_PREC_F64, 5, flush, ctypes.byref(s), ctypes.byref(g),
                               ctypes.c_void_p(work.data_ptr()), b1.value, q._stream_ptr()) == 0
        assert s.value > 0 and g.value > 0
    assert L.qr_step1_time(64, 8, q.QR_PREC_F64, 5, 1, ctypes.byref(s), ctypes.byref(g),
                           ctypes.c_void_p(work.data_ptr()), b0.value, q._stream_ptr()) == -7
    shapes = [(256, 256), (512, 512)]
    res, tab, log = _run(q, shapes, tmp_path, q.QR_PREC_F32, "f", flush=True)
    assert tab["step1"] == "multcallflushlru"
    assert len([e for e in log if e["kind"] == 5]) == len(tuning.grid_pairs())
    assert not [e for e in log if e["kind"] == 1]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    pre, out, guided = _replay_guided(log, shapes, sms, 1, step1_kind=5)
    assert guided == 0
    entries = {(e["m"], e["n"]): (e["nb"], e["ib"]) for e in tab["entries"]}
    assert entries == {s_: v[1] for s_, v in out.items()}
