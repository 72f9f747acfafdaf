"""Measured task costs for the runtime's ticket order.

The persistent kernel runs its tasks in a ticket order computed on the host
by list scheduling (earliest free worker, longest remaining path first). The
order is only as good as the task costs it assumes: with flop counts the
panel tasks (GEQRT, TSQRT), whose level-2 parts run far below the update's
rate, look cheaper than they are, and CTAs take tickets for tasks whose
panels are not done yet. In the paper's empirical spirit the costs are
measured instead: for each (NB, IB) of a tuning table one factorization of
an order-N matrix is traced (qr_set_trace) and the median service time of
each task type becomes its cost (qr_set_task_costs). A second traced run
with those costs installed refines them. The result is written to a JSON file
that the package installs at first use.

    python -m paper_1102_5328_gb300.calibrate --table paper_1102_5328_gb300/tuned/gb300_fp64.json \
        --out paper_1102_5328_gb300/tuned/gb300_fp64_costs.json

Orchestration only: every traced run is qr_factor_d/_s.
"""
import argparse
import json
import os
import sys

import numpy as np
import torch

from . import lib, qr_factor, qr_set_task_costs, qr_set_trace, read_trace

TYPES = ("GEQRT", "UNMQR", "TSQRT", "TSMQR")


def measure(n, nb, ib, dtype, seed=7):
    """Median service time (us) per task type of one traced flat-tree
    factorization of an n x n uniform[-0.5, 0.5) matrix, and the run's
    wall time (ms) from the trace."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    A0 = (torch.rand(n, n, device="cuda", generator=g, dtype=dtype) - 0.5).t()
    ntasks = lib().qr_task_count(n, n, nb, ib)
    buf = torch.zeros((ntasks, 4), dtype=torch.int64, device="cuda")
    A = A0.clone()
    qr_factor(A, nb, ib, p=1)  # warm-up, builds the ticket order
    A = A0.clone()
    torch.cuda.synchronize()
    qr_set_trace(buf)
    try:
        qr_factor(A, nb, ib, p=1)
        torch.cuda.synchronize()
    finally:
        qr_set_trace(None)
    _, typ, _, _, t_ready, t_done = read_trace(buf, ntasks)
    svc = (t_done - t_ready) / 1e3
    costs = [float(np.median(svc[typ == t])) for t in range(4)]
    return costs, [int((typ == t).sum()) for t in range(4)], float(t_done.max()) / 1e6


def calibrate(table, passes=2, n_cap=10000):
    with open(table) as f:
        tab = json.load(f)
    dtype = torch.float32 if tab.get("prec") == "fp32" else torch.float64
    # each distinct flat-tree pair, at the largest square order it was chosen for
    pairs = {}
    for e in tab["entries"]:
        if e.get("p", 1) == 1 and e["m"] == e["n"]:
            k = (e["nb"], e["ib"])
            pairs[k] = max(pairs.get(k, 0), e["n"])
    out = []
    for (nb, ib), n in sorted(pairs.items()):
        n = min(n, n_cap)
        qr_set_task_costs(dtype, nb, ib, None)
        runs = []
        for _ in range(passes):
            costs, counts, ms = measure(n, nb, ib, dtype)
            runs.append({"costs_us": costs, "span_ms": ms})
            qr_set_task_costs(dtype, nb, ib, costs)
        out.append({"nb": nb, "ib": ib, "n": n, "costs": runs[-1]["costs_us"], "counts": counts, "passes": runs})
    return {"prec": "fp32" if dtype == torch.float32 else "fp64", "types": list(TYPES), "entries": out}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--table", required=True)
    ap.add_argument("--out", required=True)
    ap.add_argument("--passes", type=int, default=2)
    ap.add_argument("--n-cap", type=int, default=10000)
    a = ap.parse_args(argv)
    torch.cuda.set_device(0)
    res = calibrate(a.table, a.passes, a.n_cap)
    s = json.dumps(res, indent=1)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    with open(a.out, "w") as f:
        f.write(s + "\n")
    print(s)
    return 0


if __name__ == "__main__":
    sys.exit(main())
