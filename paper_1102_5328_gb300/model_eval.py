"""What the learned cost model gains inside the empirical search, measured on
the GB300: the PSPAYG search with and without the model (qr_tune use_model =
0 / k on the same shapes), judged by an exhaustive search over the whole
(NB, IB) grid on the same kernels.

    python -m paper_1102_5328_gb300.model_eval --es es.jsonl --es-held es_held.jsonl \
        --plain pspayg.jsonl --plain-run pspayg_run.json --plain-table pspayg.json \
        --model pspayg_model.jsonl --model-run pspayg_model_run.json --model-table pspayg_model.json \
        --out paper_1102_5328_gb300/tuned/gb300_fp64_model_eval.json

Reported, per search: wall seconds (total, Step 1, Step 2, model fitting),
factorizations timed, and per shape the ratio P(choice) / P(grid best),
where P comes from the exhaustive log at that shape (flat tree) and the
choice is
  * the search's own table entry (nearest tuned shape, Sec. 6.1) -- for the
    tuned orders and the held-out shapes;
  * for the model search also the model's own proposal (qr_model_propose)
    on the held-out shapes, which no search timed.
The exhaustive wall time at the tuned orders is measured (its run JSON) and
also projected to the paper's 6 runs per point (6 x the per-point medians).
"""
import argparse
import ctypes
import json
import os
import sys

import numpy as np

from . import lib
from .tune_eval import flops, load_log, nearest_shape


def _run_json(path):
    with open(path) as f:
        return json.loads(f.read().strip().splitlines()[-1])


def _shapes(spec):
    out = []
    for s in spec.split(","):
        if s:
            if "x" in s:
                m, n = s.lower().split("x")
                out.append((int(m), int(n)))
            else:
                out.append((int(s), int(s)))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--es", required=True, help="exhaustive-search log over the tuned orders")
    ap.add_argument("--es-held", default="", help="exhaustive-search log over the held-out shapes")
    ap.add_argument("--es-run", default="", help="JSON printed by the exhaustive run over the tuned orders")
    for w in ("plain", "model"):
        ap.add_argument("--%s" % w, required=True, help="log of the %s search" % w)
        ap.add_argument("--%s-run" % w, required=True)
        ap.add_argument("--%s-table" % w, required=True)
    ap.add_argument("--tuned", default="1000,2000,4000,6000,8000,10000")
    ap.add_argument("--heldout", default="2700,4200,5000,30000x1000")
    ap.add_argument("--out", default="")
    ap.add_argument("--shared-step1", action="store_true",
                    help="the model search reused the plain search's Step-1 timings: charge it the same Step 1")
    a = ap.parse_args(argv)

    _, es = load_log(a.es)
    if a.es_held:
        es.update(load_log(a.es_held)[1])
    tuned, held = _shapes(a.tuned), _shapes(a.heldout)

    def grid_at(shape):
        c = {(k[2], k[3]): flops(*shape) / v[0] / 1e9 for k, v in es.items() if (k[0], k[1]) == shape}
        if not c:
            raise SystemExit("no exhaustive timings at %s" % (shape,))
        best = max(c, key=lambda p: c[p])
        return c, best

    res = {"source": {k: os.path.basename(getattr(a, k)) for k in ("es", "es_held", "plain", "model")},
           "tuned": ["%dx%d" % s for s in tuned], "heldout": ["%dx%d" % s for s in held]}
    L = lib()
    work = None
    for w in ("plain", "model"):
        run = _run_json(getattr(a, w + "_run"))
        with open(getattr(a, w + "_table")) as f:
            tab = json.load(f)
        decision = {(e["m"], e["n"]): (e["nb"], e["ib"]) for e in tab["entries"]}
        rows = []
        for shape in tuned + held:
            c, best = grid_at(shape)
            choice = decision[nearest_shape(shape, list(decision))]
            row = {"shape": "%dx%d" % shape, "heldout": shape in held, "grid_best": list(best),
                   "grid_best_gflops": c[best], "choice": list(choice), "ratio": c[choice] / c[best]}
            if w == "model" and shape in held:
                import torch
                if work is None:
                    work = torch.empty(4 << 20, dtype=torch.uint8, device="cuda")
                L.qr_clear_tables()
                assert L.qr_load_table(getattr(a, w + "_table").encode()) == 0
                nb, ib, sec = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
                rc = L.qr_model_propose(shape[0], shape[1], 0, ctypes.byref(nb), ctypes.byref(ib), ctypes.byref(sec),
                                        ctypes.c_void_p(work.data_ptr()), work.numel(), None)
                assert rc == 0, rc
                prop = (nb.value, ib.value)
                row.update({"model_proposal": list(prop), "model_predicted_s": sec.value,
                            "model_proposal_ratio": c[prop] / c[best]})
            rows.append(row)
        ratios = [r["ratio"] for r in rows]
        if w == "model" and a.shared_step1:
            run = dict(run)
            run["step1_seconds"] = res["plain"]["step1_seconds"]
            run["seconds"] = run["seconds"] + run["step1_seconds"]
        res[w] = {"seconds": run["seconds"], "step1_seconds": run["step1_seconds"],
                  "step2_seconds": run["step2_seconds"], "model_seconds": run.get("model_seconds", 0.0),
                  "factorizations_timed": run["factorizations_timed"], "model_fallbacks": run.get("model_fallbacks", 0),
                  "mean_ratio": float(np.mean(ratios)), "min_ratio": float(np.min(ratios)),
                  "optimum_found": "%d/%d" % (sum(r["choice"] == r["grid_best"] for r in rows), len(rows)),
                  "per_shape": rows}
        if w == "model":
            pr = [r["model_proposal_ratio"] for r in rows if "model_proposal_ratio" in r]
            res[w]["heldout_proposal_mean_ratio"] = float(np.mean(pr)) if pr else None
            res[w]["heldout_proposal_min_ratio"] = float(np.min(pr)) if pr else None
    # the exhaustive search's cost at the tuned orders
    es_tuned = [v[0] for k, v in es.items() if (k[0], k[1]) in tuned]
    res["full_grid_seconds_6reps_projection"] = float(6 * sum(es_tuned))
    if a.es_run:
        ej = _run_json(a.es_run)
        res["es_measured_seconds"] = ej["seconds"]
        res["es_reps"] = ej["reps"]
    for w in ("plain", "model"):
        res[w]["over_full_grid_6reps"] = res[w]["seconds"] / res["full_grid_seconds_6reps_projection"]
    res["model_saves_step2_seconds"] = res["plain"]["step2_seconds"] - res["model"]["step2_seconds"]
    res["model_saves_total_fraction"] = 1.0 - res["model"]["seconds"] / res["plain"]["seconds"]
    s = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s + "\n")
    print(s)
    return 0


if __name__ == "__main__":
    sys.exit(main())
