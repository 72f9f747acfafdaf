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

`--report N,NB,IB` prints per-type service and wait times and the busy
fraction of the persistent CTAs over the run of one traced factorization
(`--flop-weights` first removes the measured costs of that pair).

Orchestration only: every traced run is qr_factor_d/_s.
"""
import argparse
import json
import os
import sys

import numpy as np
import torch

from . import lib, qr_factor, qr_set_task_costs, qr_set_trace, qr_task_count, read_trace

TYPES = ("GEQRT", "UNMQR", "TSQRT", "TSMQR")


def trace_run(n, nb, ib, dtype, seed=7):
    """One traced flat-tree factorization of an n x n uniform[-0.5, 0.5)
    matrix (after an untraced warm-up): read_trace's arrays."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    A0 = (torch.rand(n, n, device="cuda", generator=g, dtype=dtype) - 0.5).t()
    ntasks = qr_task_count(n, n, nb, ib, dtype)
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
    return read_trace(buf, ntasks)


def measure(n, nb, ib, dtype, seed=7):
    """Median service time (us) per task type of one traced factorization,
    the task counts, and the run's span (ms) from the trace."""
    _, typ, _, _, t_ready, t_done = trace_run(n, nb, ib, dtype, seed)
    svc = (t_done - t_ready) / 1e3
    costs = [float(np.median(svc[typ == t])) for t in range(4)]
    return costs, [int((typ == t).sum()) for t in range(4)], float(t_done.max()) / 1e6


def report(n, nb, ib, dtype, workers, bins=10):
    """Per task type: count, median/p90 service and wait (us), share of the
    workers' time; and the fraction of worker slots busy in each tenth of
    the run."""
    _, typ, _, t_take, t_ready, t_done = trace_run(n, nb, ib, dtype)
    span = float(t_done.max())
    rows = []
    for t in range(4):
        sel = typ == t
        svc = (t_done - t_ready)[sel] / 1e3
        wt = (t_ready - t_take)[sel] / 1e3
        rows.append({"type": TYPES[t], "count": int(sel.sum()), "service_med_us": float(np.median(svc)),
                     "service_p90_us": float(np.percentile(svc, 90)), "wait_med_us": float(np.median(wt)),
                     "share": float(svc.sum() * 1e3 / (span * workers))})
    busy = busy_fractions(t_ready, t_done, workers, bins)
    return {"n": n, "nb": nb, "ib": ib, "span_ms": span / 1e6, "types": rows, "busy_per_tenth": busy.round(3).tolist()}


def busy_fractions(t_start, t_end, workers, bins=10):
    """Fraction of `workers` slots busy in each of `bins` equal parts of
    [0, max(t_end)], given each task's busy interval [t_start, t_end)."""
    t_start = np.asarray(t_start, dtype=np.float64)
    t_end = np.asarray(t_end, dtype=np.float64)
    edges = np.linspace(0.0, float(t_end.max()), bins + 1)
    busy = np.zeros(bins)
    for k in range(bins):
        lo, hi = edges[k], edges[k + 1]
        busy[k] = np.clip(np.minimum(t_end, hi) - np.maximum(t_start, lo), 0, None).sum() / (workers * (hi - lo))
    return busy


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
    ap.add_argument("--table", help="tuning table whose flat-tree pairs are calibrated")
    ap.add_argument("--out", help="cost file to write")
    ap.add_argument("--passes", type=int, default=2)
    ap.add_argument("--n-cap", type=int, default=10000)
    ap.add_argument("--report", default="", help="N,NB,IB: print a trace report of one factorization instead")
    ap.add_argument("--prec", choices=["f64", "f32"], default="f64")
    ap.add_argument("--flop-weights", action="store_true", help="report: clear measured costs first")
    a = ap.parse_args(argv)
    torch.cuda.set_device(0)
    if a.report:
        n, nb, ib = (int(v) for v in a.report.split(","))
        dtype = torch.float32 if a.prec == "f32" else torch.float64
        lib()
        if a.flop_weights:
            qr_set_task_costs(dtype, nb, ib, None)
        workers = 2 * torch.cuda.get_device_properties(0).multi_processor_count
        print(json.dumps(report(n, nb, ib, dtype, workers), indent=1))
        return 0
    if not a.table or not a.out:
        ap.error("--table and --out are required unless --report is given")
    res = calibrate(a.table, a.passes, a.n_cap)
    s = json.dumps(res, indent=1)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    with open(a.out, "w") as f:
        f.write(s + "\n")
    print(s)
    return 0


if __name__ == "__main__":
    sys.exit(main())
