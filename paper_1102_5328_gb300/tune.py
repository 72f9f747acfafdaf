"""Command-line driver of the install-time tuner (qr_tune in the C library).

    python -m paper_1102_5328_gb300.tune --mode pspayg --heuristic 2 \
        --ns 1000,2000,4000,6000,8000,10000 --reps 6 \
        --table paper_1102_5328_gb300/tuned/gb300_fp64.json --log tune_pspayg.jsonl

--mode pspayg: Step 1 (TSMQR kernel benchmark over the 119-pair grid),
Properties 5.1/5.2 and Heuristic H0/H1/H2, then Step 2 with prune-as-you-go
(Secs. 5–6 of the paper). --mode es: exhaustive search (every grid pair at
every shape). --flush: Step 1 as MultCallFlushLRU instead of No Flush.
--use-model K: the learned cost model ranks the survivors from the third
order on and only the K fastest-predicted are timed (see qr_tune).
--sm-budgets B1,B2,...: Step 2 once per SM budget (QR_OPT_SM_BUDGET, the GPU
counterpart of the paper's core counts, Sec. 6.1; 0 = the whole GPU), one
log shared by all budgets (Step 1 runs once), the tables merged into --table.
Shapes come from --ns (square) and --shapes (m x n list).
Prints one JSON line with the wall times the library measured.
"""
import argparse
import ctypes
import json
import os
import sys

import torch

from . import _lib, lib, QR_PREC_F32, QR_PREC_F64


def parse_shapes(ns, shapes):
    out = []
    if ns:
        out += [(int(v), int(v)) for v in ns.split(",") if v]
    if shapes:
        for s in shapes.split(","):
            if s:
                m, n = s.lower().split("x")
                out.append((int(m), int(n)))
    return out


def write_table(path, tab):
    """A decision table in the layout qr_load_table reads: one entry per line,
    keys in the library's order."""
    head = {k: v for k, v in tab.items() if k != "entries"}
    lines = ["{"] + ["  %s: %s," % (json.dumps(k), json.dumps(v)) for k, v in head.items()]
    lines.append('  "entries": [')
    ents = [json.dumps({k: e[k] for k in ("m", "n", "nb", "ib", "p", "gflops", "sms") if k in e})
            for e in tab["entries"]]
    lines.append(",\n".join("    " + e for e in ents))
    lines += ["  ]", "}"]
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def run(shapes, mode, heuristic, reps, prec, table, log, stream=None, use_model=0, flush=False, ib_tol=0):
    from . import QR_OPT_TUNE_IB_TOL, qr_get_option, qr_set_option
    old_tol = qr_get_option(QR_OPT_TUNE_IB_TOL)
    qr_set_option(QR_OPT_TUNE_IB_TOL, int(ib_tol))
    try:
        return _run(shapes, mode, heuristic, reps, prec, table, log, stream, use_model, flush, ib_tol)
    finally:
        qr_set_option(QR_OPT_TUNE_IB_TOL, old_tol)


def _run(shapes, mode, heuristic, reps, prec, table, log, stream, use_model, flush, ib_tol):
    L = lib()
    max_m = max(m for m, _ in shapes)
    max_n = max(n for _, n in shapes)
    # workspace must cover the largest m and the largest n at once
    need = 0
    for m, n in shapes:
        b = ctypes.c_int64()
        _lib.check(L.qr_tune_workspace(m, n, prec, ctypes.byref(b)), "qr_tune_workspace")
        need = max(need, b.value)
    work = torch.empty(need, dtype=torch.uint8, device="cuda")
    k = len(shapes)
    ms = (ctypes.c_int64 * k)(*[m for m, _ in shapes])
    nn = (ctypes.c_int64 * k)(*[n for _, n in shapes])
    secs = (ctypes.c_double * 6)()
    s = stream if stream is not None else torch.cuda.current_stream()
    code = (1 if mode == "es" else 0) | (2 if flush else 0)
    rc = L.qr_tune(ms, nn, k, heuristic, code, int(use_model), reps, prec, (table or "").encode(),
                   (log or "").encode(), ctypes.c_void_p(work.data_ptr()), need, secs, ctypes.c_void_p(s.cuda_stream))
    _lib.check(rc, "qr_tune")
    return {"mode": mode, "heuristic": heuristic, "reps": reps, "use_model": int(use_model),
            "step1": "multcallflushlru" if flush else "noflush", "ib_tol_permille": int(ib_tol),
            "shapes": shapes, "seconds": secs[0],
            "step1_seconds": secs[1], "step2_seconds": secs[2], "factorizations_timed": int(secs[3]),
            "model_seconds": secs[4], "model_fallbacks": int(secs[5]),
            "table": table, "log": log, "max_m": max_m, "max_n": max_n}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--mode", choices=["pspayg", "es"], default="pspayg")
    ap.add_argument("--heuristic", type=int, default=2)
    ap.add_argument("--ns", default="1000,2000,4000,6000,8000,10000")
    ap.add_argument("--shapes", default="")
    ap.add_argument("--reps", type=int, default=6)
    ap.add_argument("--prec", choices=["f64", "f32"], default="f64")
    ap.add_argument("--table", default="")
    ap.add_argument("--log", default="")
    ap.add_argument("--use-model", type=int, default=0)
    ap.add_argument("--flush", action="store_true")
    ap.add_argument("--sm-budgets", default="", help="comma-separated SM budgets (0 = whole GPU)")
    ap.add_argument("--ib-tol", type=int, default=0,
                    help="Step 1: keep, per preselected NB, every IB within this many 1/1000 of its best IB's rate")
    a = ap.parse_args(argv)
    if a.table:
        os.makedirs(os.path.dirname(os.path.abspath(a.table)), exist_ok=True)
    prec = QR_PREC_F32 if a.prec == "f32" else QR_PREC_F64
    shapes = parse_shapes(a.ns, a.shapes)
    if not a.sm_budgets:
        res = run(shapes, a.mode, a.heuristic, a.reps, prec, a.table, a.log, use_model=a.use_model, flush=a.flush,
                  ib_tol=a.ib_tol)
        print(json.dumps(res))
        return 0
    from . import QR_OPT_SM_BUDGET, qr_set_option
    merged, runs = None, []
    try:
        for b in [int(v) for v in a.sm_budgets.split(",") if v]:
            qr_set_option(QR_OPT_SM_BUDGET, b)
            tb = (a.table or "tune_table.json") + ".sms%d" % b
            r = run(shapes, a.mode, a.heuristic, a.reps, prec, tb, a.log, use_model=a.use_model, flush=a.flush,
                    ib_tol=a.ib_tol)
            r["sm_budget"] = b
            runs.append(r)
            t = json.load(open(tb))
            if merged is None:
                merged = t
            else:
                merged["entries"] += t["entries"]
            os.remove(tb)
    finally:
        qr_set_option(QR_OPT_SM_BUDGET, 0)
    merged["sm_budgets"] = [r["sm_budget"] for r in runs]
    merged["seconds"] = sum(r["seconds"] for r in runs)
    merged.pop("model", None)  # one model per budget run; not merged
    if a.table:
        write_table(a.table, merged)
        lib().qr_load_table(a.table.encode())
    print(json.dumps({"runs": runs, "table": a.table}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
