"""Pins for oracle/tuning.py (CPU only): hand-built hulls with known
selections, brute-force hull membership, the paper's interpolation example,
and the guarantee of prune-as-you-go on monotone tables."""
import itertools
import os
import random

import pytest

from oracle import tuning

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_grid_counts():
    pairs = tuning.grid_pairs()
    per_nb = {}
    for nb, ib in pairs:
        per_nb[nb] = per_nb.get(nb, 0) + 1
    # divisors of NB in [8, NB/2], counted by hand for NB = 64, 96, ..., 512
    assert [per_nb[nb] for nb in range(64, 513, 32)] == [3, 6, 4, 7, 8, 7, 5, 12, 9, 8, 10, 8, 9, 17, 6]
    assert len(pairs) == 119
    assert (288, 9) in pairs and (480, 15) in pairs and (512, 256) in pairs and (64, 64) not in pairs


def test_prune_ib_keeps_best_per_nb():
    perf = {(64, 8): 1.0, (64, 16): 3.0, (64, 32): 2.0, (96, 8): 5.0, (96, 12): 5.0}
    assert tuning.prune_ib(perf) == {64: (16, 3.0), 96: (8, 5.0)}


def _brute_upper_hull(points):
    """Vertices of the upper hull by definition: a point is kept iff it lies
    strictly above every chord between a point on its left and one on its
    right (plus the two extreme x)."""
    pts = sorted(set(points))
    out = []
    for k, p in enumerate(pts):
        if k == 0 or k == len(pts) - 1:
            out.append(p)
            continue
        ok = True
        for a in pts[:k]:
            for b in pts[k + 1:]:
                y = a[1] + (b[1] - a[1]) * (p[0] - a[0]) / (b[0] - a[0])
                if p[1] <= y:
                    ok = False
        if ok:
            out.append(p)
    return out


@pytest.mark.parametrize("seed", range(20))
def test_upper_hull_brute_force(seed):
    rng = random.Random(seed)
    xs = rng.sample(range(64, 513, 32), rng.randint(2, 15))
    pts = [(x, rng.uniform(0, 10) + x / 100.0) for x in xs]
    assert tuning.upper_hull(pts) == _brute_upper_hull(pts)


def test_hand_built_hull_and_heuristics():
    # concave rising-then-flat curve plus points below it
    pts = {(64, 8): 2.0, (96, 8): 3.5, (128, 16): 4.5, (160, 16): 5.0, (192, 32): 5.3,
           (224, 32): 5.4, (256, 32): 5.45, (288, 32): 5.2, (320, 32): 3.0}
    hull = tuning.upper_hull([(nb, p) for (nb, _), p in pts.items()])
    # 288 (5.2) lies above the chord 256 -> 320 (4.225 at 288), so it stays
    assert [h[0] for h in hull] == [64, 96, 128, 160, 192, 224, 256, 288, 320]
    st = tuning.steepness(hull)
    # origin -> 64: 2/64; 64 -> 96: 1.5/32; 96 -> 128: 1/32; ...
    assert st[0] == pytest.approx(2.0 / 64)
    assert st[1] == pytest.approx(1.5 / 32)
    assert st[-1] < 0
    assert tuning.heuristic0(hull) == [64, 96, 128, 160, 192, 224, 256, 288, 320]
    # H1 with 3 picks: steepest segments end at 96 (0.047), 64 (0.031), 128 (0.031)
    assert tuning.heuristic1(hull, max_sel=3) == [64, 96, 128]
    # H2 with 4 iso-segments of [64, 320] (width 64): [64,128) -> 96,
    # [128,192) -> 128, [192,256) -> 192, [256,320] -> 256
    assert tuning.heuristic2(hull, 64, 320, max_sel=8, nseg=4) == [96, 128, 192, 256]


def test_preselect_returns_best_ib():
    perf = {(64, 8): 2.0, (64, 16): 2.2, (96, 8): 3.5, (96, 32): 3.0, (128, 16): 4.5, (128, 64): 4.6}
    sel = tuning.preselect(perf, heuristic=0)
    assert sel == [(64, 16), (96, 8), (128, 64)]


def test_payg_prunes_exactly_dominated():
    surv = [(64, 8), (96, 8), (128, 16), (160, 16)]
    perf = {(64, 8): 3.0, (96, 8): 4.0, (128, 16): 3.5, (160, 16): 3.9}
    # 64 < 96 with 4.0 > 3.0 -> drop 64; 128 < 160 with 3.9 > 3.5 -> drop 128;
    # 96 is beaten by nobody larger (3.5, 3.9 < 4.0) -> kept
    assert tuning.payg_prune(surv, perf) == [(96, 8), (160, 16)]
    # ties are kept
    assert tuning.payg_prune([(64, 8), (96, 8)], {(64, 8): 1.0, (96, 8): 1.0}) == [(64, 8), (96, 8)]


@pytest.mark.parametrize("seed", range(10))
def test_payg_never_loses_optimum_on_monotone_tables(seed):
    """If Property 6.1 holds for the table, PSPAYG finds the same optimum as
    measuring every preselected pair at every N (brute force)."""
    rng = random.Random(seed)
    nbs = sorted(rng.sample(range(64, 513, 32), 6))
    pairs = [(nb, 8) for nb in nbs]
    ns = [1000, 2000, 4000, 6000, 8000, 10000]
    # P(NB, N) = a_NB * N - b_NB with larger NB having larger slope and
    # larger offset: crossings only from small NB to large NB as N grows,
    # which is exactly Property 6.1
    a = {nb: 1.0 + k * 0.2 for k, nb in enumerate(nbs)}
    b = {nb: 300.0 * k * k for k, nb in enumerate(nbs)}

    def measure(n, pr):
        return a[pr[0]] * n - b[pr[0]]

    for nb1, nb2 in itertools.product(nbs, nbs):
        if nb1 > nb2:
            for i, n in enumerate(ns):
                if measure(n, (nb1, 8)) > measure(n, (nb2, 8)):
                    assert all(measure(n2, (nb1, 8)) > measure(n2, (nb2, 8)) for n2 in ns[i:])
    table, count = tuning.step2_payg(ns, pairs, measure)
    for n in ns:
        brute = max(pairs, key=lambda pr: measure(n, pr))
        assert table[n][0] == brute
    assert count <= len(pairs) * len(ns)


def test_interpolation_example_from_paper():
    g = {}
    with open(os.path.join(GOLDEN, "interpolation_example.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                g[k] = [int(x) for x in v]
    n, c = g["query"]
    assert (tuning.nearest(n, g["grid_N"]), tuning.nearest(c, g["grid_cores"])) == tuple(g["expect"])
    assert tuning.nearest(1500, [1000, 2000]) == 1000  # tie -> smaller


def test_widen_ib_keeps_the_ibs_within_tolerance():
    """The IB-tolerance extension of Property 5.1: tol = 0 is the paper's rule
    (the best IB only); a pair enters when its rate is at least (1 - tol)
    times the best IB's of the same NB, after that pair, ascending IB."""
    perf = {(64, 8): 100.0, (64, 16): 101.0, (64, 32): 90.0, (128, 8): 200.0, (128, 16): 150.0}
    pre = [(64, 16), (128, 8)]
    assert tuning.widen_ib(perf, pre, 0.0) == pre
    assert tuning.widen_ib(perf, pre, 0.0099) == pre  # 100 < 0.9901 * 101
    assert tuning.widen_ib(perf, pre, 0.02) == [(64, 16), (64, 8), (128, 8)]
    assert tuning.widen_ib(perf, pre, 0.11) == [(64, 16), (64, 8), (64, 32), (128, 8)]
    assert tuning.widen_ib(perf, pre, 0.3) == [(64, 16), (64, 8), (64, 32), (128, 8), (128, 16)]
