"""Oracle of the paper's empirical tuning rules -- TEST INFRASTRUCTURE ONLY.

Plain Python restatement, from the paper's text, of the decisions the
library's C++ tuner makes. Only tests/ (and bench.py's CPU baseline) use it.

  * the search grid of (NB, IB) pairs;
  * Property 5.1 (orthogonal pruning): per NB keep the IB with the best
    Step-1 kernel performance (Sec. 5);
  * Property 5.2 (convex hull) and Heuristic 0: the points of the upper
    convex hull of the (NB, performance) data set (Sec. 5);
  * Heuristic 1: hull points after the steepest segments, at most 8;
  * Heuristic 2: split the NB axis into iso-segments and keep the hull point
    of maximum steepness in each, at most 8 (Sec. 5);
  * Property 6.1 and prune-as-you-go (PSPAYG): after benchmarking order N,
    drop every NB2 for which a larger surviving NB1 already performs better
    (Sec. 6.3);
  * interpolation: an untuned request uses the closest benchmarked point
    (Sec. 6.1).

Readings where the paper is silent:
upper hull taken left to right with both end points, collinear middle points
dropped; steepness of a hull point = slope of the hull segment that ends at
it, the leftmost point's segment starting at the origin; Heuristic 1 sorts
by steepness, ties to the smaller NB; Heuristic 2 uses nseg equal-width
intervals over [min NB, max NB] of the data set, the last one closed, empty
intervals contributing nothing; PAYG removes on strict inequality only;
nearest-point ties go to the smaller value.
"""


def grid_pairs(nb_min=64, nb_max=512, nb_step=32, ib_min=8):
    """All (NB, IB) with NB in nb_min..nb_max step nb_step and IB a divisor
    of NB with ib_min <= IB <= NB/2."""
    out = []
    for nb in range(nb_min, nb_max + 1, nb_step):
        for ib in range(ib_min, nb // 2 + 1):
            if nb % ib == 0:
                out.append((nb, ib))
    return out


def prune_ib(perf):
    """Property 5.1. perf: {(NB, IB): P}. Returns {NB: (IB, P)} keeping, per
    NB, the IB of highest P (ties: smaller IB)."""
    best = {}
    for (nb, ib), p in sorted(perf.items()):
        if nb not in best or p > best[nb][1]:
            best[nb] = (ib, p)
    return best


def _cross(o, a, b):
    return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])


def upper_hull(points):
    """Upper convex hull of [(x, y)], left to right, both end points kept,
    collinear middle points dropped (monotone chain)."""
    pts = sorted(set(points))
    hull = []
    for p in pts:
        while len(hull) >= 2 and _cross(hull[-2], hull[-1], p) >= 0:
            hull.pop()
        hull.append(p)
    return hull


def steepness(hull):
    """Slope of the hull segment ending at each hull point (origin for the
    first point)."""
    out = []
    prev = (0.0, 0.0)
    for p in hull:
        out.append((p[1] - prev[1]) / (p[0] - prev[0]))
        prev = p
    return out


def heuristic0(hull):
    return [p[0] for p in hull]


def heuristic1(hull, max_sel=8):
    st = steepness(hull)
    order = sorted(range(len(hull)), key=lambda i: (-st[i], hull[i][0]))
    return sorted(hull[i][0] for i in order[:max_sel])


def heuristic2(hull, nb_lo, nb_hi, max_sel=8, nseg=8):
    st = steepness(hull)
    width = (nb_hi - nb_lo) / float(nseg)
    chosen = []
    for s in range(nseg):
        a = nb_lo + s * width
        b = nb_lo + (s + 1) * width
        best = None
        for i, p in enumerate(hull):
            inside = (a <= p[0] < b) or (s == nseg - 1 and p[0] == nb_hi)
            if inside and (best is None or st[i] > st[best]):
                best = i
        if best is not None:
            chosen.append(hull[best][0])
    return sorted(chosen)[:max_sel]


def preselect(perf, heuristic=2, max_sel=8, nseg=8):
    """Step 1 decisions: Property 5.1, the hull, then H0/H1/H2. Returns the
    preselected [(NB, IB)] sorted by NB."""
    best = prune_ib(perf)
    pts = [(nb, best[nb][1]) for nb in best]
    hull = upper_hull(pts)
    nbs = [nb for nb, _ in perf]
    if heuristic == 0:
        sel = heuristic0(hull)
    elif heuristic == 1:
        sel = heuristic1(hull, max_sel)
    else:
        sel = heuristic2(hull, min(nbs), max(nbs), max_sel, nseg)
    return [(nb, best[nb][0]) for nb in sel]


def widen_ib(perf, pre, tol):
    """An extension of Property 5.1 (the paper keeps only the best IB per NB;
    tol = 0 is that rule): each preselected (NB, IB*) also brings every other
    IB of that NB whose Step-1 rate is at least (1 - tol) times IB*'s, in
    ascending IB after IB*, so that Step 2 decides between IBs the kernel
    benchmark cannot tell apart. pre: preselect()'s list."""
    out = []
    for nb, ib0 in pre:
        out.append((nb, ib0))
        if tol <= 0:
            continue
        p0 = perf[(nb, ib0)]
        out += [(nb, ib) for (n2, ib) in sorted(perf) if n2 == nb and ib != ib0 and perf[(nb, ib)] >= (1.0 - tol) * p0]
    return out


def payg_prune(survivors, perf_n):
    """Property 6.1 (PSPAYG). survivors: [(NB, IB)]; perf_n: {(NB, IB): P}
    at the order just benchmarked. Keeps a pair unless a pair with larger NB
    has strictly higher P."""
    keep = []
    for nb2, ib2 in survivors:
        dominated = any(nb1 > nb2 and perf_n[(nb1, ib1)] > perf_n[(nb2, ib2)] for nb1, ib1 in survivors)
        if not dominated:
            keep.append((nb2, ib2))
    return keep


def step2_payg(order_ns, survivors, measure):
    """Step 2 with PSPAYG: for each N ascending, measure every surviving pair
    (measure(N, pair) -> P), record the best, then prune. Returns
    ({N: (pair, P)}, number of measurements)."""
    table, count = {}, 0
    surv = list(survivors)
    for n in sorted(order_ns):
        perf_n = {}
        for pr in surv:
            perf_n[pr] = measure(n, pr)
            count += 1
        best = max(surv, key=lambda pr: (perf_n[pr], -pr[0]))
        table[n] = (best, perf_n[best])
        surv = payg_prune(surv, perf_n)
    return table, count


def nearest(value, grid):
    """Closest grid value (ties: the smaller one), Sec. 6.1 interpolation."""
    return min(grid, key=lambda g: (abs(g - value), g))
