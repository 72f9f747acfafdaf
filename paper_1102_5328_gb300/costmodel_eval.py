"""Train the MLP cost model on the tuner's own timings and measure what it
gains on held-out shapes.

    python -m paper_1102_5328_gb300.costmodel_eval --es es.jsonl --table gb300_fp64.json \
        --out paper_1102_5328_gb300/tuned/gb300_fp64_costmodel.json

Training data: every logged factorization time at the training shapes
(square tuned orders and the tall-skinny shapes) -> features
(log m, log n, NB/512, IB/256), target log(seconds). Held-out shapes: the
off-grid squares and a tall-skinny shape never trained on. For each
held-out shape three choices are compared against the best measured pair
(regret = 1 - P(choice) / P(best)):
  * the method without the model: the closest tuned shape's pair (Sec. 6.1);
  * the model alone: argmin of predicted time over the grid;
  * the model as a pruner: measure only its top-k pairs, keep the fastest
    (k measurements instead of the whole preselection).
"""
import argparse
import json
import os
import sys

import numpy as np

from . import costmodel, inputs
from .tune_eval import flops, load_log, nearest_shape


def parse(shapes):
    out = []
    for s in shapes.split(","):
        if not s:
            continue
        if "x" in s:
            m, n = s.split("x")
            out.append((int(m), int(n)))
        else:
            out.append((int(s), int(s)))
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--es", required=True)
    ap.add_argument("--table", required=True)
    ap.add_argument("--train", default="1000,2000,4000,6000,8000,10000,20000x500,100000x256,50000x2000")
    ap.add_argument("--heldout", default="2700,4200,5000,30000x1000")
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--topk", type=int, default=3)
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--out", default="")
    a = ap.parse_args(argv)

    _, es = load_log(a.es)
    with open(a.table) as f:
        tab = json.load(f)
    decision = {(e["m"], e["n"]): (e["nb"], e["ib"]) for e in tab["entries"]}
    train = parse(a.train)
    held = parse(a.heldout)
    pts = [(k, v[0]) for k, v in es.items() if (k[0], k[1]) in train]
    F = costmodel.features([p[0][0] for p in pts], [p[0][1] for p in pts], [p[0][2] for p in pts],
                           [p[0][3] for p in pts])
    y = np.log(np.array([p[1] for p in pts]))
    model = costmodel.CostModel(inputs.mlp_init(a.seed))
    Z = model.standardize(F, fit=True)
    ymean = float(y.mean())
    final_loss = model.train(Z, y - ymean, a.steps, a.lr)

    rows = []
    for shape in held:
        cands = {(k[2], k[3]): flops(*shape) / v[0] / 1e9 for k, v in es.items() if (k[0], k[1]) == shape}
        pairs = sorted(cands)
        best = max(pairs, key=lambda p: cands[p])
        Fh = costmodel.features([shape[0]] * len(pairs), [shape[1]] * len(pairs), [p[0] for p in pairs],
                                [p[1] for p in pairs])
        pred = model.forward(model.standardize(Fh)) + ymean
        order = np.argsort(pred)
        model_choice = pairs[int(order[0])]
        topk = [pairs[int(i)] for i in order[: a.topk]]
        topk_choice = max(topk, key=lambda p: cands[p])
        near = decision[nearest_shape(shape, list(decision))]
        meas_logt = np.log(np.array([flops(*shape) / (cands[p] * 1e9) for p in pairs]))
        rows.append({
            "m": shape[0], "n": shape[1], "best": list(best), "best_gflops": cands[best],
            "nearest_table_choice": list(near), "regret_nearest": 1 - cands[near] / cands[best],
            "model_choice": list(model_choice), "regret_model": 1 - cands[model_choice] / cands[best],
            "model_topk": [list(p) for p in topk], "regret_model_topk": 1 - cands[topk_choice] / cands[best],
            "rmse_log_time": float(np.sqrt(np.mean((pred - meas_logt) ** 2))),
            "pairs": len(pairs),
        })
    res = {
        "train_shapes": [list(s) for s in train], "heldout_shapes": [list(s) for s in held],
        "train_samples": len(pts), "steps": a.steps, "lr": a.lr, "final_train_mse": final_loss,
        "topk": a.topk,
        "mean_regret_nearest": float(np.mean([r["regret_nearest"] for r in rows])),
        "mean_regret_model": float(np.mean([r["regret_model"] for r in rows])),
        "mean_regret_model_topk": float(np.mean([r["regret_model_topk"] for r in rows])),
        "per_shape": rows,
    }
    s = json.dumps(res, indent=1)
    if a.out:
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        with open(a.out, "w") as f:
            f.write(s + "\n")
    print(s)
    return 0


if __name__ == "__main__":
    sys.exit(main())
