"""Per-size-class tile shapes for the batched QR, chosen empirically.

The paper's tuner picks (NB, IB) per matrix order N (Sec. 6.1); for a batch
of small uneven matrices the analogue is a choice per size class of the row
count m. For each class the batch's own matrices of that class are factored
with every candidate pair (one persistent launch per candidate, median of a
few runs, CUDA events), and the fastest pair is installed with
qr_batched_set_class. Orchestration only: every timed launch is
qr_factor_batched_d/_s.
"""
import json
import statistics

import numpy as np
import torch

from . import BatchedPlan, qr_batched_set_class, qr_flops

CLASSES = (64, 128, 256, 512)
CANDIDATES = ((32, 8), (32, 16), (64, 8), (64, 16), (64, 32), (128, 8), (128, 16), (128, 32), (256, 8), (256, 16),
              (512, 8), (512, 16), (512, 32))


def _time(plan, src_flat, work_flat, reps):
    ts = []
    for _ in range(reps + 1):
        work_flat.copy_(src_flat)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.launch()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts[1:])


def tune_classes(mats, dtype=torch.float64, reps=3, candidates=CANDIDATES, classes=CLASSES, install=True):
    """mats: list of NumPy matrices (the batch). Returns {m_hi: {...}}."""
    out = {}
    lo = 0
    for hi in classes:
        sub = [a for a in mats if lo < a.shape[0] <= hi]
        lo = hi
        if not sub:
            continue
        sizes = [a.size for a in sub]
        offs = np.concatenate([[0], np.cumsum([(s + 31) // 32 * 32 for s in sizes])])
        flat = np.zeros(int(offs[-1]))
        for a, o in zip(sub, offs[:-1]):
            flat[int(o):int(o) + a.size] = np.ascontiguousarray(a.T).reshape(-1)
        src = torch.from_numpy(flat).to(dtype).cuda()
        work = src.clone()
        views = [work[int(o):int(o) + a.size].view(a.shape[1], a.shape[0]).t() for o, a in zip(offs[:-1], sub)]
        fl = sum(qr_flops(*a.shape) for a in sub)
        res = {}
        for nb, ib in candidates:
            if ib > nb:
                continue
            plan = BatchedPlan(views, nb, ib)
            ms = _time(plan, src, work, reps)
            res["%d,%d" % (nb, ib)] = {"ms": ms, "gflops": fl / (ms * 1e-3) / 1e9}
        best = max(res, key=lambda k: res[k]["gflops"])
        nb, ib = map(int, best.split(","))
        if install:
            qr_batched_set_class(dtype, hi, nb, ib)
        out[hi] = {"count": len(sub), "best": [nb, ib], "gflops": res[best]["gflops"], "candidates": res}
    return out


if __name__ == "__main__":
    import argparse

    from . import inputs

    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    ms, ns = inputs.batch_shapes(a.count, seed=4)
    mats = inputs.batch_matrices(ms, ns, seed=5)
    res = {}
    for dt, name in ((torch.float64, "f64"), (torch.float32, "f32")):
        r = tune_classes(mats, dt, a.reps)
        res[name] = {str(k): {"count": v["count"], "best": v["best"], "gflops": v["gflops"]} for k, v in r.items()}
    s = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s + "\n")
    print(s)
