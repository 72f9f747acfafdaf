"""Benchmark of the FP64 tile Householder QR on one GB300 (or N replicas).

Workload: square FP64 tile QR of order N = 10000 (the largest order of the
paper's Step-2 discretization, Sec. 6.1), entries uniform[-0.5, 0.5) from a
seed, with the (NB, IB) pair of the tuning table (or --nb/--ib).
A step = restore A from a pristine device copy, then qr_factor_d (layout
conversion, the persistent DAG kernel, conversion back). Inputs (800 MB)
are larger than L2, so no flush is needed between steps.

Metric: GFlop/s = (2mn^2 - 2n^3/3) / t (= 4/3 N^3 / t, the paper's P of
Sec. 2.2, independent of IB). With --gpus N > 1 (torchrun, one rank per GPU)
every rank factors its own matrix (replicas: a single factorization does not
shard), value = total credited flops / max over ranks of the time.

--impl reference times the CPU oracle (unblocked Householder QR, OpenMP) on
the host cores on a bounded sample of the same workload: the first K
reflectors of the same N = 10000 matrix.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_DEFAULT = 10000
SEED = 10000

# DRAM bytes (read + write) of one persistent_qr<double> launch, carried over
# from one ncu capture of the same configuration and kernel sources
# (profiles/persistent_qr_fp64_n10000.md), not measured by this run; None for
# any other configuration.
TRAFFIC_BYTES = {(10000, 10000, 128, 8): 57.57e9 + 41.40e9}
TRAFFIC_SOURCE = ("ncu capture of this kernel and configuration (dram__bytes_read.sum + dram__bytes_write.sum, "
                  "profiles/persistent_qr_fp64_n10000.md), not measured in this run")


def max_over_ranks(x, device="cuda"):
    """The maximum of a per-rank float over all ranks (the job takes as long
    as its slowest rank); the value itself with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gflops(flops_per_step, steps, ranks, max_ms):
    """GFLOP/s of the whole job: every rank factors its own matrix (replicas),
    so the credited flops add up over ranks; the time is the slowest rank's."""
    return flops_per_step * steps * ranks / (max_ms * 1e-3) / 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_sample(A_np, seconds_target=15.0):
    """Time the oracle's first k reflectors of A (fp64, OpenMP on the host
    cores). Returns (GFlop/s, k, seconds, threads)."""
    import oracle
    threads = oracle.set_threads(0)
    m, n = A_np.shape

    def flops(k):
        return sum(4.0 * (m - j) * (n - j - 1) + 2.0 * (m - j - 1) for j in range(k))

    k = 16
    t0 = time.perf_counter()
    oracle.geqr2(A_np, kmax=k)
    dt = time.perf_counter() - t0
    rate = flops(k) / max(dt, 1e-9)
    k2 = 16
    while k2 < n and flops(k2 * 2) / rate < seconds_target:
        k2 *= 2
    t0 = time.perf_counter()
    oracle.geqr2(A_np, kmax=k2)
    dt = time.perf_counter() - t0
    return flops(k2) / dt / 1e9, k2, dt, threads


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    from paper_1102_5328_gb300 import inputs
    import oracle
    n = args.n
    A_np = inputs.uniform_matrix(n, n, seed=SEED)
    threads = oracle.set_threads(0)
    m = n

    def flops(k):
        return sum(4.0 * (m - j) * (n - j - 1) + 2.0 * (m - j - 1) for j in range(k))

    # size one step to ~8 s of CPU work
    t0 = time.perf_counter()
    oracle.geqr2(A_np, kmax=16)
    rate = flops(16) / max(time.perf_counter() - t0, 1e-9)
    k = 16
    while k < n and flops(k * 2) / rate < 8.0:
        k *= 2
    for _ in range(args.warmup):
        oracle.geqr2(A_np, kmax=k)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.geqr2(A_np, kmax=k)
        times.append(time.perf_counter() - t0)
    T = sum(times)
    value = flops(k) * args.steps / T / 1e9
    sample = "first %d Householder reflectors of the N=%d uniform[-0.5,0.5) matrix per step" % (k, n)
    line = {
        "impl": "reference", "metric": "QR GFlop/s (2mn^2 - 2n^3/3)/t", "value": value, "unit": "GFLOP/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "fp64 square tile QR, N=%d, uniform[-0.5,0.5)" % n, "m": n, "n": n},
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_batched(args):
    """Batched uneven QR: 4096 matrices, m ~ U{32..512}, n ~ U{16..m}, N(0,1),
    one persistent launch captured in a CUDA graph with the input restore,
    replayed; GFLOP/s = sum of credited flops / median replay time."""
    import torch

    import paper_1102_5328_gb300 as q
    from paper_1102_5328_gb300 import inputs

    torch.cuda.set_device(0)
    out = {}
    ms, ns = inputs.batch_shapes(args.count, seed=4)
    mats = inputs.batch_matrices(ms, ns, seed=5)
    total_flops = float(sum(q.qr_flops(int(m), int(n)) for m, n in zip(ms, ns)))
    sizes = [int(m) * int(n) for m, n in zip(ms, ns)]
    offs = np.concatenate([[0], np.cumsum([(sz + 31) // 32 * 32 for sz in sizes])])
    flat_np = np.zeros(int(offs[-1]))
    for a, o in zip(mats, offs[:-1]):
        flat_np[int(o):int(o) + a.size] = np.ascontiguousarray(a.T).reshape(-1)
    for dt, name in ((torch.float64, "f64"), (torch.float32, "f32")):
        # all matrices in one buffer: the graph restores them with one copy
        src_flat = torch.from_numpy(flat_np).to(dt).cuda()
        work_flat = src_flat.clone()
        work = [work_flat[int(o):int(o) + int(m) * int(n)].view(int(n), int(m)).t()
                for o, m, n in zip(offs[:-1], ms, ns)]
        plan = q.BatchedPlan(work, args.nb, args.ib)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            plan.launch(stream=s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            work_flat.copy_(src_flat)
            plan.launch(stream=torch.cuda.current_stream())
        for _ in range(args.warmup):
            g.replay()
        torch.cuda.synchronize()
        times = []
        for _ in range(max(args.steps, 20)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        med = statistics.median(times)
        out[name] = {"median_ms": med, "gflops": total_flops / (med * 1e-3) / 1e9, "replays": len(times),
                     "status": plan.status()}
    nominal_fp64 = 152 * 2 * 2 * 2.070e9 / 1e12
    out["f64"]["roofline"] = {"bound": "alu", "kernel": "batched_qr<double> (FP64 DFMA pipe)",
                              "achieved": out["f64"]["gflops"] / 1e3, "peak": nominal_fp64, "unit": "TFLOP/s",
                              "frac": out["f64"]["gflops"] / 1e3 / nominal_fp64}
    nominal_fp32 = 152 * 128 * 2 * 2.070e9 / 1e12
    out["f32"]["roofline"] = {"bound": "alu", "kernel": "batched_qr<float> (FP32 FMA pipe)",
                              "achieved": out["f32"]["gflops"] / 1e3, "peak": nominal_fp32, "unit": "TFLOP/s",
                              "frac": out["f32"]["gflops"] / 1e3 / nominal_fp32}
    line = {"workload": "batched uneven QR, %d matrices, m~U{32..512}, n~U{16..m}, N(0,1)" % args.count,
            "metric": "GFLOP/s (sum of 2mn^2-2n^3/3 per replay)", "unit": "GFLOP/s",
            "credited_gflop_per_batch": total_flops / 1e9, "results": out,
            "note": "each replay restores the inputs (device copy) and runs one persistent launch"}
    if not args.no_cpu:
        import oracle
        threads = oracle.set_threads(0)
        fl, t0, k = 0.0, time.perf_counter(), 0
        while k < len(mats) and time.perf_counter() - t0 < 10.0:
            oracle.geqr2(mats[k])
            fl += q.qr_flops(*mats[k].shape)
            k += 1
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": fl / dt / 1e9, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                                "sample": "the first %d matrices of the batch, one by one (%.1f s)" % (k, dt)}
    print(json.dumps(line))
    return 0


def run_ls(args):
    """Least squares, A = U diag(sigma) V^T (16384 x 4096, kappa 1e6), 8 RHS:
    plain FP64 QR solve vs FP32 factorization + FP64 augmented refinement vs
    tensor-core (BF16x3, TF32) factorizations + FP64 GMRES-based refinement;
    forward error against the oracle's doubled-precision refined solution.
    Also the factorization alone at each low precision (CUDA events)."""
    import torch

    import paper_1102_5328_gb300 as q
    from paper_1102_5328_gb300 import inputs

    torch.cuda.set_device(0)
    m, n, k = args.ls_m, args.ls_n, 8
    A_np, B_np = inputs.ls_problem(m, n, k, kappa=1e6, seed=5)
    A = torch.from_numpy(np.ascontiguousarray(A_np.T)).cuda().t()
    B = torch.from_numpy(np.ascontiguousarray(B_np.T)).cuda().t()
    names = {"fp64": ("fp64", q.QR_PREC_F64, 0, 0), "fp32": ("mixed_fp32_ir", q.QR_PREC_F32, 50, 1),
             "fp32_gmres": ("mixed_fp32_gmres_ir", q.QR_PREC_F32, 50, 2),
             "bf16x3": ("mixed_bf16x3_gmres_ir", q.QR_PREC_BF16X3, 20, 2),
             "tf32": ("mixed_tf32_gmres_ir", q.QR_PREC_TF32, 20, 2)}
    res = {}
    for key in args.ls_precs.split(","):
        name, prec, it, refine = names[key]
        q.qr_set_option(q.QR_OPT_LS_REFINE, refine)
        dt = torch.float64 if prec == q.QR_PREC_F64 else torch.float32
        nb, ib, pd = q.qr_lookup_p(m, n, dt)
        if args.nb:
            nb, ib = args.nb, args.ib
        pd = args.ls_p if args.ls_p else pd
        tol = args.ls_tol if prec != q.QR_PREC_F64 else 2.0 ** -52
        # every solve at the faster of a few configurations, all reported:
        # the factorization table's (NB, IB, p); the same pair with the
        # library's domain count (p = 0: ceil(MT / NT), shorter Q-application
        # chains); and, when the table's tiles are larger than 64, NB = 64
        # with the same IB (the few-column Q applications stage 64-row tiles
        # whole)
        cands = [(nb, ib, pd)]
        if not args.nb and not args.ls_p:
            cands.append((nb, ib, 0))
            if nb > 64:
                cands.append((64, ib, 0))
        labels = ["table", "p_default", "nb64"]
        for ci, (nb_c, ib_c, p_c) in enumerate(cands):
            X, info = q.qr_solve_ls(A, B, prec=prec, nb=nb_c, ib=ib_c, max_iter=it, tol=tol, p=p_c)  # warm-up
            torch.cuda.synchronize()
            ts = []
            for _ in range(max(args.steps, 3)):
                t0 = time.perf_counter()
                X, info = q.qr_solve_ls(A, B, prec=prec, nb=nb_c, ib=ib_c, max_iter=it, tol=tol, p=p_c)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            r = {"median_s": statistics.median(ts), "info": list(info), "nb": nb_c, "ib": ib_c, "p": p_c, "tol": tol,
                 "refine": ["none", "augmented", "gmres"][refine] if prec != q.QR_PREC_F64 else "none",
                 "X": X.cpu().numpy()}
            if len(cands) > 1:
                res["%s_%s" % (name, labels[ci])] = dict(r)
            if name not in res or r["median_s"] < res[name]["median_s"]:
                res[name] = r
    q.qr_set_option(q.QR_OPT_LS_REFINE, 0)
    # the FP32-storage factorization alone, FP32 cores vs tensor cores
    fac = {}
    nb, ib, pd = q.qr_lookup_p(m, n, torch.float32)
    A32 = torch.from_numpy(np.ascontiguousarray(A_np.T.astype(np.float32))).cuda().t()
    for pname, prec in (("fp32", q.QR_PREC_F32), ("tf32", q.QR_PREC_TF32), ("bf16x3", q.QR_PREC_BF16X3)):
        W = A32.clone()
        f = q.qr_factor_mixed(W, prec, nb, ib, pd)
        ms = []
        for _ in range(max(args.steps, 3)):
            W.copy_(A32)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            q.qr_factor_mixed(W, prec, nb, ib, pd, T=f.T, scratch=f.scratch)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        fac[pname] = {"median_ms": statistics.median(ms), "gflops": q.qr_flops(m, n) / statistics.median(ms) / 1e6,
                      "nb": nb, "ib": ib, "p": pd, "status": f.status()}
    line = {"workload": "least squares %dx%d, kappa 1e6, %d RHS N(0,1)" % (m, n, k), "metric": "seconds per solve"}
    if not args.no_cpu:
        import oracle
        threads = oracle.set_threads(0)
        t0 = time.perf_counter()
        Xref, its = oracle.ls_refine(A_np, B_np, maxit=30)
        line["cpu_baseline"] = {"value": time.perf_counter() - t0, "unit": "s per solve", "cores": threads,
                                "kind": "oracle",
                                "sample": "full problem: fp64 Householder QR solve + doubled-precision refinement"}
        for name in res:
            X = res[name].pop("X")
            fe = np.linalg.norm(X - Xref, axis=0) / np.linalg.norm(Xref, axis=0)
            res[name]["forward_error_max"] = float(fe.max())
            res[name]["forward_error"] = [float(v) for v in fe]
        line["oracle_refinement_iterations"] = its
    else:
        for name in res:
            res[name].pop("X")
    line["results"] = res
    line["factorization"] = fac
    if "fp64" in res and "mixed_fp32_ir" in res:
        line["speedup_mixed_over_fp64"] = res["fp64"]["median_s"] / res["mixed_fp32_ir"]["median_s"]
    print(json.dumps(line))
    return 0


def run_cholesky(args):
    """FP64 tile Cholesky (chol_factor_d) of an SPD matrix of order --n
    (G G^T / n + I), nb from the Cholesky tuning table (or --nb): GFLOP/s
    credited n^3 / 3, CUDA events around each call (layout conversions
    included); the persistent kernel's share against the FP64 FMA peak; the
    CPU oracle's column Cholesky on a bounded sample (order 3000)."""
    import ctypes

    import torch

    import paper_1102_5328_gb300 as q
    from paper_1102_5328_gb300 import inputs

    torch.cuda.set_device(0)
    n = args.n
    A_np = inputs.spd_matrix(n, seed=n)
    A0 = torch.from_numpy(np.ascontiguousarray(A_np.T)).cuda().t()
    A = A0.clone()
    nb = args.nb
    if not nb:
        v = ctypes.c_int()
        q.lib().chol_lookup(n, ctypes.byref(v))
        nb = v.value
    f = q.chol_factor(A, nb)
    ms = []
    for s in range(args.warmup + args.steps):
        A.copy_(A0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        q.chol_factor(A, nb, scratch=f.scratch)
        e1.record()
        torch.cuda.synchronize()
        if s >= args.warmup:
            ms.append(e0.elapsed_time(e1))
    st = f.status()
    flops = float(n) ** 3 / 3.0
    med = statistics.median(ms)
    peak_live = q.qr_peak_fp64()
    nominal_peak = 152 * 2 * 2 * 2.070e9 / 1e9
    line = {"workload": "fp64 tile Cholesky, N=%d, SPD G G^T/n + I" % n, "metric": "Cholesky GFlop/s (n^3/3)/t",
            "value": flops / (med * 1e-3) / 1e9, "unit": "GFLOP/s", "ms_per_step": med, "steps": args.steps,
            "nb": nb, "status": list(st), "tasks": int(q.lib().chol_task_count_n(n, nb)),
            "roofline": {"bound": "alu", "peak": nominal_peak, "unit": "GFLOP/s",
                         "frac": flops / (med * 1e-3) / 1e9 / nominal_peak,
                         "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                         "peak_measured_live": peak_live}}
    if not args.no_cpu:
        import oracle
        threads = oracle.set_threads(0)
        ns = 3000
        S = inputs.spd_matrix(ns, seed=ns)
        t0 = time.perf_counter()
        oracle.potrf(S)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": ns ** 3 / 3.0 / dt / 1e9, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                                "sample": "column Cholesky of an SPD matrix of order %d (%.1f s)" % (ns, dt)}
    print(json.dumps(line))
    return 0


def run_lu(args):
    """FP64 tile LU with incremental pivoting (lu_factor_d) of a uniform
    [-0.5, 0.5) matrix of order --n, nb from the LU tuning table (or --nb): GFLOP/s credited
    2 n^3 / 3, CUDA events around each call (layout conversions included),
    against the FP64 FMA peak; the CPU oracle's task-by-task tile LU on a
    bounded sample (order 1000)."""
    import torch

    import paper_1102_5328_gb300 as q
    from paper_1102_5328_gb300 import inputs

    torch.cuda.set_device(0)
    n = args.n
    A_np = inputs.uniform_matrix(n, n, seed=n)
    A0 = torch.from_numpy(np.ascontiguousarray(A_np.T)).cuda().t()
    A = A0.clone()
    nb = args.nb
    if not nb:
        import ctypes
        v = ctypes.c_int()
        q.lib().lu_lookup(n, ctypes.byref(v))
        nb = v.value
    f = q.lu_factor(A, nb)
    ms = []
    for s in range(args.warmup + args.steps):
        A.copy_(A0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        q.lu_factor(A, nb, piv=f.piv, scratch=f.scratch)
        e1.record()
        torch.cuda.synchronize()
        if s >= args.warmup:
            ms.append(e0.elapsed_time(e1))
    st = f.status()
    flops = 2.0 * float(n) ** 3 / 3.0
    med = statistics.median(ms)
    peak_live = q.qr_peak_fp64()
    nominal_peak = 152 * 2 * 2 * 2.070e9 / 1e9
    line = {"workload": "fp64 tile LU (incremental pivoting), N=%d, uniform[-0.5,0.5)" % n,
            "metric": "LU GFlop/s (2n^3/3)/t", "value": flops / (med * 1e-3) / 1e9, "unit": "GFLOP/s",
            "ms_per_step": med, "steps": args.steps, "nb": nb, "status": list(st),
            "tasks": int(q.lib().lu_task_count_n(n, nb)),
            "roofline": {"bound": "alu", "peak": nominal_peak, "unit": "GFLOP/s",
                         "frac": flops / (med * 1e-3) / 1e9 / nominal_peak,
                         "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                         "peak_measured_live": peak_live}}
    if not args.no_cpu:
        from oracle import lu
        ns = 1000
        S = inputs.uniform_matrix(ns, ns, seed=ns)
        t0 = time.perf_counter()
        lu.getrf_incpiv(S, nb)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 2.0 * ns ** 3 / 3.0 / dt / 1e9, "unit": "GFLOP/s", "cores": 1,
                                "kind": "oracle",
                                "sample": "tile LU of order %d, NB %d, NumPy row operations (%.1f s)" % (ns, nb, dt)}
    print(json.dumps(line))
    return 0


def run_step1(args):
    """The Step-1 kernel benchmark (Sec. 5) for one (NB, IB): a batch of
    2 x SMs independent TSMQR tasks per launch, No Flush; GFLOP/s credits
    4 NB^3 per task."""
    import ctypes

    import torch

    import paper_1102_5328_gb300 as q

    torch.cuda.set_device(0)
    L = q.lib()
    nb, ib = args.nb or 128, args.ib or 8
    prec = {"f64": 0, "f32": 1, "tf32": 2, "bf16x3": 3}[args.prec]
    b = ctypes.c_int64()
    q._lib.check(L.qr_step1_workspace(nb, prec, 0, ctypes.byref(b)), "qr_step1_workspace")
    work = torch.empty(b.value, dtype=torch.uint8, device="cuda")
    s, g = ctypes.c_double(), ctypes.c_double()
    for _ in range(max(1, args.warmup)):
        q._lib.check(L.qr_step1_time(nb, ib, prec, 3, 0, ctypes.byref(s), ctypes.byref(g),
                                     ctypes.c_void_p(work.data_ptr()), b.value, q._stream_ptr()), "qr_step1_time")
    q._lib.check(L.qr_step1_time(nb, ib, prec, max(args.steps, 3), 0, ctypes.byref(s), ctypes.byref(g),
                                 ctypes.c_void_p(work.data_ptr()), b.value, q._stream_ptr()), "qr_step1_time")
    peak = q.qr_peak_fp64()
    line = {"workload": "Step-1 TSMQR batch, %s, NB=%d IB=%d" % (args.prec, nb, ib), "ms_per_launch": s.value * 1e3,
            "gflops": g.value}
    if prec == 0:
        line.update({"fp64_peak_live_gflops": peak, "frac_of_live_peak": g.value / peak})
    else:
        fp32_peak = 152 * 128 * 2 * 2.070  # GFLOP/s: 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz
        line.update({"fp32_peak_derived_gflops": fp32_peak, "frac_of_fp32_peak": g.value / fp32_peak})
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--nb", type=int, default=0)
    ap.add_argument("--ib", type=int, default=0)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--prec", default="f64", choices=["f64", "f32", "tf32", "bf16x3"],
                    help="step1: precision of the TSMQR batch (tf32 / bf16x3: FP32 tiles, tensor-core products)")
    ap.add_argument("--workload", default="qr", choices=["qr", "batched", "ls", "step1", "cholesky", "lu"],
                    help="qr: the headline line; batched / ls: the extension workloads (own JSON lines)")
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--ls-m", type=int, default=16384)
    ap.add_argument("--ls-n", type=int, default=4096)
    ap.add_argument("--ls-tol", type=float, default=1e-11,
                    help="mixed solve: stop once ||dx|| <= tol ||x|| (FP64-level accuracy for kappa 1e6)")
    ap.add_argument("--ls-p", type=int, default=0, help="panel domains of the solve's factorization (0 = the tuned table's p)")
    ap.add_argument("--ls-precs", default="fp64,fp32,bf16x3",
                    help="least-squares solves to time: fp64, fp32 (augmented IR), fp32_gmres, bf16x3, tf32 (GMRES-IR)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "ls":
        return run_ls(args)
    if args.workload == "step1":
        return run_step1(args)
    if args.workload == "lu":
        return run_lu(args)
    if args.workload == "cholesky":
        return run_cholesky(args)

    import torch
    import torch.distributed as dist

    import paper_1102_5328_gb300 as q
    from paper_1102_5328_gb300 import inputs

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")

    def barrier():
        if ws > 1:
            dist.barrier()

    n = args.n
    m = n
    nb, ib = (args.nb, args.ib) if args.nb else q.qr_lookup(m, n, torch.float64)
    A_np = inputs.uniform_matrix(m, n, seed=SEED + rank)
    A0 = torch.from_numpy(np.ascontiguousarray(A_np.T)).cuda().t()  # column-major, on device
    A = A0.clone().t().contiguous().t()
    t_elems, sbytes = q.qr_workspace(m, n, nb, ib, torch.float64)
    T = torch.empty(t_elems, dtype=torch.float64, device="cuda")
    scratch = torch.empty(sbytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    lib = q.lib()

    def step():
        A.copy_(A0)
        q.qr_factor(A, nb, ib, T=T, scratch=scratch, stream=stream)

    peak_live = q.qr_peak_fp64()
    q.qr_set_option(q.QR_OPT_RECORD_EVENTS, 1)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = q.qr_status(scratch)
    if st != 0:
        raise RuntimeError("device status %d after warm-up" % st)

    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    kernel_ms = []
    ev0.record(stream)
    for _ in range(args.steps):
        step()
        kernel_ms.append(None)
    ev1.record(stream)
    torch.cuda.synchronize()
    total_ms = ev0.elapsed_time(ev1)
    # per-launch kernel time of the dominant (persistent) kernel: re-time
    # each step with the library's own events on the launching stream
    for s in range(args.steps):
        step()
        kernel_ms[s] = q.qr_last_kernel_ms()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    total_ms = max_over_ranks(total_ms)
    flops = q.qr_flops(m, n)
    value = whole_job_gflops(flops, args.steps, ws, total_ms)
    kavg = sum(kernel_ms) / len(kernel_ms)
    nominal_peak = 152 * 2 * 2 * 2.070e9 / 1e12  # TFLOP/s: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
    achieved = flops / (kavg * 1e-3) / 1e12
    roofline = {
        "bound": "alu", "kernel": "persistent_qr<double> (FP64 DFMA pipe)",
        "achieved": achieved, "peak": nominal_peak, "unit": "TFLOP/s", "frac": achieved / nominal_peak,
        "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
        "peak_measured_live": peak_live / 1e3, "frac_of_measured": achieved / (peak_live / 1e3),
        "traffic": TRAFFIC_BYTES.get((m, n, nb, ib)), "kernel_ms_avg": kavg,
    }
    if roofline["traffic"] is not None:
        roofline["traffic_source"] = TRAFFIC_SOURCE

    e2e = None
    if not args.no_e2e:
        # end to end through the public API: pinned host A -> device, factor,
        # factored A and T -> host, every step
        hA = torch.from_numpy(np.ascontiguousarray(A_np.T)).pin_memory()
        hOut = torch.empty_like(hA).pin_memory()
        hT = torch.empty(t_elems, dtype=torch.float64).pin_memory()
        Ad = A  # reuse the device buffer (column-major view)

        def e2e_step():
            Ad.t().copy_(hA, non_blocking=True)
            q.qr_factor(Ad, nb, ib, T=T, scratch=scratch, stream=stream)
            hOut.copy_(Ad.t(), non_blocking=True)
            hT.copy_(T, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ks = max(2, min(args.steps, 3))
        ea.record(stream)
        for _ in range(ks):
            e2e_step()
        eb.record(stream)
        torch.cuda.synchronize()
        ems = ea.elapsed_time(eb)
        ems = max_over_ranks(ems)
        e2e = {"value": whole_job_gflops(flops, ks, ws, ems), "unit": "GFLOP/s",
               "h2d_bytes_per_step": 8 * m * n, "d2h_bytes_per_step": 8 * m * n + 8 * t_elems,
               "steps": ks}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        g, k, dt, threads = cpu_oracle_sample(A_np)
        cpu = {"value": g, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
               "sample": "first %d Householder reflectors of the same N=%d matrix (%.1f s)" % (k, n, dt)}

    # the tuner's own figures: NOT measured by this run; copied from the
    # committed install-time tuning campaign (paper_1102_5328_gb300.tune /
    # tune_eval on a GB300), with the repetitions behind each figure
    tuning = None
    tpath = os.path.join(ROOT, "paper_1102_5328_gb300", "tuned", "gb300_fp64_reliability.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tj = json.load(f)
        tuning = {k: tj.get(k) for k in ("autotuned_over_grid_best", "autotuned_over_grid_best_min",
                                        "optimum_found", "tuning_seconds", "full_grid_seconds",
                                        "full_grid_seconds_basis", "tuning_over_full_grid",
                                        "tuning_seconds_tuned_orders", "tuning_over_full_grid_tuned_orders",
                                        "tuned_orders_basis", "heuristic", "ib_tol_permille", "use_model",
                                        "es_reps", "pspayg_reps", "model")}
        tuning = {k: v for k, v in tuning.items() if v is not None}
        tuning["source"] = "committed: paper_1102_5328_gb300/tuned/gb300_fp64_reliability.json (not this run)"
        mpath = os.path.join(ROOT, "paper_1102_5328_gb300", "tuned", "gb300_fp64_model_eval.json")
        if os.path.exists(mpath):
            with open(mpath) as f:
                mj = json.load(f)
            tuning["with_model"] = {
                "tuning_seconds": mj["model"]["seconds"], "plain_tuning_seconds": mj["plain"]["seconds"],
                "autotuned_over_grid_best": mj["model"]["mean_ratio"],
                "autotuned_over_grid_best_min": mj["model"]["min_ratio"],
                "heldout_proposal_over_grid_best": mj["model"].get("heldout_proposal_mean_ratio"),
                "factorizations_timed": mj["model"]["factorizations_timed"],
                "plain_factorizations_timed": mj["plain"]["factorizations_timed"],
                "source": "committed: paper_1102_5328_gb300/tuned/gb300_fp64_model_eval.json (not this run)"}

    if rank == 0:
        line = {
            "metric": "QR GFlop/s (2mn^2 - 2n^3/3)/t", "value": value, "unit": "GFLOP/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "fp64 square tile QR, N=%d, uniform[-0.5,0.5)" % n, "m": m, "n": n,
                       "nb": nb, "ib": ib, "l2": "inputs (800 MB) larger than L2; no flush",
                       "parallelism": "replicas" if ws > 1 else "1 GPU"},
            "pct_fp64_peak": 100.0 * value / ws / (nominal_peak * 1e3),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": 3 * args.steps, "clocks": clk, "tuning": tuning,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
