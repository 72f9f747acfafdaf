"""Command-line driver of the install-time tuner (qr_tune in the C library).

    python -m paper_1102_5328_gb300.tune --mode pspayg --heuristic 2 \
        --ns 1000,2000,4000,6000,8000,10000 --reps 6 \
        --table paper_1102_5328_gb300/tuned/gb300_fp64.json --log tune_pspayg.jsonl

--mode pspayg: Step 1 (TSMQR kernel benchmark over the 119-pair grid),
Properties 4.1/4.2 and Heuristic H0/H1/H2, then Step 2 with prune-as-you-go
(Secs. 4-5 of the paper). --mode es: exhaustive search (every grid pair at
every shape). --flush: Step 1 as MultCallFlushLRU instead of No Flush.
--use-model K: the learned cost model ranks the survivors from the third
order on and only the K fastest-predicted are timed (see qr_tune).
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


def run(shapes, mode, heuristic, reps, prec, table, log, stream=None, use_model=0, flush=False):
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
            "step1": "multcallflushlru" if flush else "noflush", "shapes": shapes, "seconds": secs[0],
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
    a = ap.parse_args(argv)
    if a.table:
        os.makedirs(os.path.dirname(os.path.abspath(a.table)), exist_ok=True)
    res = run(parse_shapes(a.ns, a.shapes), a.mode, a.heuristic, a.reps,
              QR_PREC_F32 if a.prec == "f32" else QR_PREC_F64, a.table, a.log, use_model=a.use_model, flush=a.flush)
    print(json.dumps(res))
    return 0


if __name__ == "__main__":
    sys.exit(main())
