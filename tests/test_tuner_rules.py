"""The C++ tuner's decision rules (host-only entry points of libtileqr.so)
against the Python oracle of the paper's rules, on random tables. CPU only:
these calls make no GPU call."""
import ctypes
import json
import os
import random

import pytest

from oracle import tuning

lib_mod = pytest.importorskip("paper_1102_5328_gb300._lib")


@pytest.fixture(scope="module")
def L():
    return lib_mod.load()


def _ia(xs):
    return (ctypes.c_int * len(xs))(*xs)


def _da(xs):
    return (ctypes.c_double * len(xs))(*xs)


def test_grid_matches(L):
    n = L.qr_tune_grid(64, 512, 32, 8, 0, None, None)
    nb = (ctypes.c_int * n)()
    ib = (ctypes.c_int * n)()
    assert L.qr_tune_grid(64, 512, 32, 8, n, nb, ib) == n
    assert list(zip(nb, ib)) == tuning.grid_pairs()


@pytest.mark.parametrize("heur", [0, 1, 2])
@pytest.mark.parametrize("seed", range(15))
def test_preselect_matches_oracle(L, heur, seed):
    rng = random.Random(seed * 3 + heur)
    pairs = tuning.grid_pairs()
    # a rising, saturating kernel curve with noise, different per IB
    perf = {(nb, ib): (1.0 - 2.0 ** (-nb / 150.0)) * (1.0 - 0.3 * ib / nb) + rng.uniform(-0.08, 0.08)
            for nb, ib in pairs}
    if seed % 3 == 0:  # sometimes a non-monotone curve
        perf = {k: v + 0.2 * ((k[0] // 32) % 3 == 0) for k, v in perf.items()}
    want = tuning.preselect(perf, heuristic=heur)
    nb = [p[0] for p in pairs]
    ib = [p[1] for p in pairs]
    out_nb = (ctypes.c_int * 32)()
    out_ib = (ctypes.c_int * 32)()
    k = L.qr_tune_preselect(len(pairs), _ia(nb), _ia(ib), _da([perf[p] for p in pairs]), heur, 8, 8, out_nb, out_ib)
    got = list(zip(out_nb[:k], out_ib[:k]))
    assert got == want
    if heur:
        assert len(got) <= 8


@pytest.mark.parametrize("seed", range(20))
def test_payg_matches_oracle(L, seed):
    rng = random.Random(seed)
    nbs = sorted(rng.sample(range(64, 513, 32), rng.randint(1, 8)))
    surv = [(nb, 8) for nb in nbs]
    perf = {p: float(rng.randint(0, 5)) for p in surv}  # many ties
    want = tuning.payg_prune(surv, perf)
    keep = (ctypes.c_int * len(surv))()
    assert L.qr_tune_payg(len(surv), _ia(nbs), _da([perf[p] for p in surv]), keep) == 0
    assert [p for p, k in zip(surv, keep) if k] == want


def test_nearest_matches_oracle(L):
    grid = [1000, 2000, 4000, 6000, 8000, 10000]
    g = (ctypes.c_int64 * len(grid))(*grid)
    for v in list(range(0, 12001, 250)) + [1500, 3000, 5000, 7000, 9000]:
        assert L.qr_tune_nearest(v, g, len(grid)) == tuning.nearest(v, grid)


def test_table_roundtrip_and_lookup(L, tmp_path):
    t = {"prec": "fp64", "entries": [
        {"m": 1000, "n": 1000, "nb": 64, "ib": 16, "gflops": 100.0},
        {"m": 2000, "n": 2000, "nb": 96, "ib": 32, "gflops": 300.0},
        {"m": 10000, "n": 10000, "nb": 192, "ib": 32, "gflops": 900.0}]}
    p = tmp_path / "t.json"
    p.write_text(json.dumps(t, indent=2).replace('"m":', '"m":'))
    # the library's reader wants its own flat one-line-per-entry format
    lines = ['{', '  "prec": "fp64",', '  "entries": [']
    for i, e in enumerate(t["entries"]):
        lines.append('    {"m": %d, "n": %d, "nb": %d, "ib": %d, "gflops": %.4f}%s'
                     % (e["m"], e["n"], e["nb"], e["ib"], e["gflops"], "," if i < 2 else ""))
    lines[-1] = lines[-1].replace('{"m": 2000,', '{"m": 2000,')
    lines += ['    ,{"m": 50000, "n": 500, "nb": 64, "ib": 8, "p": 16, "gflops": 300.0}']
    lines += ['  ]', '}']
    p.write_text("\n".join(lines))
    assert L.qr_load_table(str(p).encode()) == 0
    nb, ib = ctypes.c_int(), ctypes.c_int()
    for n_req, expect in [(1800, 2000), (1400, 1000), (1500, 1000), (7000, 10000), (20000, 10000)]:
        assert L.qr_lookup(n_req, n_req, 0, ctypes.byref(nb), ctypes.byref(ib)) == 0
        e = [x for x in t["entries"] if x["n"] == tuning.nearest(n_req, [1000, 2000, 10000])][0]
        assert e["n"] == expect
        assert (nb.value, ib.value) == (e["nb"], e["ib"])
    p_ = ctypes.c_int()
    assert L.qr_lookup_p(60000, 400, 0, ctypes.byref(nb), ctypes.byref(ib), ctypes.byref(p_)) == 0
    assert (nb.value, ib.value, p_.value) == (64, 8, 16)
    assert L.qr_lookup_p(1000, 1000, 0, ctypes.byref(nb), ctypes.byref(ib), ctypes.byref(p_)) == 0
    assert p_.value == 1  # entries without p are flat-tree entries
    L.qr_clear_tables()
    assert L.qr_lookup(5000, 5000, 0, ctypes.byref(nb), ctypes.byref(ib)) == 0
    assert (nb.value, ib.value) == (128, 16)  # built-in default


def test_every_declared_symbol_is_exported(L):
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    names = set()
    for h in os.listdir(os.path.join(root, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(root, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:int|int64_t|double|void)\s+\**\s*(\w+)\s*\(", src, flags=re.M))
    assert len(names) >= 10
    for nm in sorted(names):
        assert hasattr(L, nm), nm
    declared = {s[0] for s in lib_mod.SIGNATURES}
    assert names == declared, (names ^ declared)


def test_task_costs_and_schedule_options_validate(L):
    """Host-only settings of the list schedule: measured task costs and the
    flop-weight options reject bad arguments and accept good ones."""
    good = _da([2.5, 1.8, 2.7, 2.2])
    assert L.qr_set_task_costs(0, 128, 8, good) == 0
    assert L.qr_set_task_costs(0, 128, 8, None) == 0  # removed again
    assert L.qr_set_task_costs(2, 128, 8, good) == -1
    assert L.qr_set_task_costs(0, 4, 2, good) == -2
    assert L.qr_set_task_costs(0, 128, 0, good) == -3
    assert L.qr_set_task_costs(1, 64, 16, _da([1.0, -1.0, 1.0, 1.0])) == -4
    assert L.qr_set_task_costs(1, 64, 16, _da([1.0, float("nan"), 1.0, 1.0])) == -4
    for opt, default in ((8, 150), (9, 100)):
        assert L.qr_get_option(opt) == default
        assert L.qr_set_option(opt, 5) == -2
        assert L.qr_set_option(opt, 300) == 0 and L.qr_get_option(opt) == 300
        assert L.qr_set_option(opt, default) == 0
    assert L.qr_set_trace(None, 0) == 0
    assert L.qr_set_trace(None, -1) == -2


def test_busy_fractions_of_a_trace():
    """The trace report's utilisation: two workers, a run of 10 time units
    cut in 10 bins; worker A busy over [0, 10), worker B over [5, 10)."""
    pytest.importorskip("torch")
    from paper_1102_5328_gb300.calibrate import busy_fractions
    b = busy_fractions([0, 5], [10, 10], workers=2, bins=10)
    assert b.tolist() == [0.5] * 5 + [1.0] * 5
    # tasks back to back on one worker fill it; a gap shows as idle time
    b = busy_fractions([0, 2, 6], [2, 4, 8], workers=1, bins=4)
    assert b.tolist() == [1.0, 1.0, 0.0, 1.0]


def test_task_count_follows_the_column_split(L):
    """Flat-tree task counts: per panel k one GEQRT, S chunks of UNMQR per
    trailing tile column, and per tile row below one TSQRT plus S chunks of
    TSMQR per trailing column; FP64 splits update tasks in two from NB = 128
    on, FP32 from NB = 192, and QR_OPT_SPLIT overrides both."""
    def count(MT, NT, S):
        c = 0
        for k in range(min(MT, NT)):
            c += 1 + (NT - k - 1) * S
            c += (MT - k - 1) * (1 + (NT - k - 1) * S)
        return c

    assert L.qr_task_count(1000, 1000, 128, 8, 0) == count(8, 8, 2)
    assert L.qr_task_count(1000, 1000, 128, 8, 1) == count(8, 8, 1)
    assert L.qr_task_count(1000, 900, 64, 8, 0) == count(16, 15, 1)
    assert L.qr_task_count(2000, 1000, 192, 16, 1) == count(11, 6, 2)
    assert L.qr_task_count(2000, 1000, 384, 16, 0) == count(6, 3, 4)
    assert L.qr_set_option(3, 3) == 0
    try:
        assert L.qr_task_count(1000, 1000, 64, 8, 0) == count(16, 16, 3)
    finally:
        assert L.qr_set_option(3, 0) == 0


def test_read_trace_decodes_records():
    """read_trace unpacks the 32-byte trace records (task | type | SM, and
    three globaltimer stamps made relative to the earliest ticket)."""
    torch = pytest.importorskip("torch")
    import paper_1102_5328_gb300 as q
    recs = [(5, 3, 17, 1000, 1400, 2000), (0, 0, 151, 900, 950, 1500), (7, 5, 2, 1200, 1300, 1800)]
    buf = torch.zeros((4, 4), dtype=torch.int64)
    for r, (task, typ, sm, t0, t1, t2) in enumerate(recs):
        buf[r, 0] = (sm << 48) | (typ << 40) | task
        buf[r, 1], buf[r, 2], buf[r, 3] = t0, t1, t2
    task, typ, sm, tt, tr, td = q.read_trace(buf, 3)
    assert task.tolist() == [5, 0, 7] and typ.tolist() == [3, 0, 5] and sm.tolist() == [17, 151, 2]
    assert tt.tolist() == [100, 0, 300] and tr.tolist() == [500, 50, 400] and td.tolist() == [1100, 600, 900]


def _restore_tables(L):
    """Put back the committed tuning tables (later tests may look pairs up)."""
    L.qr_clear_tables()
    tuned = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1102_5328_gb300", "tuned")
    for name in ("gb300_fp64.json", "gb300_fp32.json"):
        if os.path.exists(os.path.join(tuned, name)):
            L.qr_load_table(os.path.join(tuned, name).encode())


def _load_synthetic_table(L, tmp_path, entries, prec="fp64"):
    path = tmp_path / "t.json"
    rows = ",\n".join('    {"m": %d, "n": %d, "nb": %d, "ib": %d, "p": %d, "gflops": 1.0, "sms": %d}' % e for e in entries)
    path.write_text('{\n  "prec": "%s",\n  "entries": [\n%s\n  ]\n}\n' % (prec, rows))
    assert L.qr_load_table(str(path).encode()) == 0


def _lookup_sms(L, m, n, sms):
    nb, ib, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert L.qr_lookup_sms(m, n, 0, sms, ctypes.byref(nb), ctypes.byref(ib), ctypes.byref(p)) == 0
    return nb.value, ib.value, p.value


def test_sm_budget_lookup_is_the_papers_interpolation(L, tmp_path):
    """The (N, SM budget) table read as the paper's (N, ncores) one: the
    paper's example (N = 1800 on 5 cores -> the point tuned for N = 2000 on
    4 cores) and random queries, against oracle.tuning.nearest applied to the
    budget and then to N. Each grid point gets a distinct (nb, ib) so the
    chosen entry is identified."""
    grid_n = [500, 1000, 2000, 4000, 6000, 8000, 10000]
    grid_c = [1, 2, 4, 8, 16, 32, 48]
    ident = {}
    entries = []
    for a, n in enumerate(grid_n):
        for b, c in enumerate(grid_c):
            nb, ib = 64 + 32 * a, 8 + b
            ident[(nb, ib)] = (n, c)
            entries.append((n, n, nb, ib, 1, c))
    try:
        _load_synthetic_table(L, tmp_path, entries)
        nb, ib, _ = _lookup_sms(L, 1800, 1800, 5)
        assert ident[(nb, ib)] == (2000, 4)
        rng = random.Random(5)
        for _ in range(200):
            n, c = rng.randint(100, 12000), rng.randint(1, 60)
            nb, ib, _ = _lookup_sms(L, n, n, c)
            assert ident[(nb, ib)] == (tuning.nearest(n, grid_n), tuning.nearest(c, grid_c)), (n, c)
    finally:
        _restore_tables(L)


def test_sm_budget_lookup_with_whole_gpu_entries(L, tmp_path):
    """Entries tuned without a budget (sms 0, the whole GPU) and a request
    for the whole GPU (0) meet; a small budget takes its own entries."""
    try:
        _load_synthetic_table(L, tmp_path, [(1000, 1000, 64, 8, 1, 0), (1000, 1000, 96, 16, 1, 8),
                                            (4000, 4000, 128, 8, 1, 0)])
        assert _lookup_sms(L, 3900, 3900, 0)[:2] == (128, 8)
        assert _lookup_sms(L, 3900, 3900, 6)[:2] == (96, 16)  # budget 8 is closest; its only entry
        assert _lookup_sms(L, 900, 900, 10000)[:2] == (64, 8)  # beyond the GPU: the whole-GPU entries
    finally:
        _restore_tables(L)
