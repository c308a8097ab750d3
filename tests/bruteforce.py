"""Brute-force references used to pin the oracle (test-only; independent of oracle/ and of the
CUDA library).

* ``smi_integral``: the mutual information of eq. (mi_sum), sum_i integral P(Z=z) f(delta_i(z), r_i) dz,
  with the measurement prior P(Z=z) of eq. (measurement_prior) evaluated pointwise as a mixture
  density and the inverse sensor model delta_i(z) of eq. (inverse_sensing) applied cell by cell.
  The integral over z is taken numerically (composite Gauss-Legendre on cell-aligned panels), the
  protocol the paper uses for its ground truth (Section 5.1). Nothing here uses the closed form
  G_{k,j} or the prefix quantities C_k of the fast algorithms.
* ``exact_cells``: the cells a fixed-point ray crosses, from exact rational slab intersections.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def kl_gain(delta: float, o: float) -> float:
    """Information gain of one cell = KL(posterior || prior) of a Bernoulli cell whose odds are
    multiplied by delta (the inverse sensor model update of eq. (bayesian_filter))."""
    from scipy.special import rel_entr

    r = o / (1.0 - o)
    post = delta * r / (1.0 + delta * r)
    return float(rel_entr(post, o) + rel_entr(1.0 - post, 1.0 - o))


def _gain(delta: float, o: float) -> float:
    if o <= 0.0 or o >= 1.0 or delta == 1.0:
        return 0.0
    return kl_gain(delta, o)


def smi_integral(o, l, sigma, delta_occ, delta_emp, e0_mode=0, noise="gauss", H=0, panels=8, order=24, skip=None):
    """Numerical integration of eq. (mi_sum) on one beam (o[n], l[n+1]).

    noise="gauss": P(z|e_j) = N(mu_j, sigma), mu_j the centre of cell j.
    noise="uniform": P(z|e_j) = U[l_j - H, l_{j+1} + H] (Theorem 4's model, unit cells).
    e0_mode=1 adds the no-return event with centre l_1 - 1/2 (or support [l_1 - 1 - H, l_1 + H]).
    A measurement outside [l_1, l_{n+1}) carries no information.
    skip: cells left out of the sum over i of eq. (mi_sum) (they still shape P(Z=z)).
    """
    skip = set() if skip is None else {i for i, v in enumerate(skip) if v}
    o = [float(v) for v in o]
    l = [float(v) for v in l]
    n = len(o)
    # first-hit probabilities from the independence model, term by term
    pe = []
    for j in range(n):
        p = o[j]
        for i in range(j):
            p *= 1.0 - o[i]
        pe.append(p)
    p0 = 1.0
    for i in range(n):
        p0 *= 1.0 - o[i]
    comps = []  # (weight, centre-or-interval)
    for j in range(n):
        comps.append((pe[j], j))
    if e0_mode:
        comps.append((p0, -1))

    def density(z):
        tot = np.zeros_like(z)
        for w, j in comps:
            if noise == "gauss":
                mu = (l[0] - 0.5) if j < 0 else 0.5 * (l[j] + l[j + 1])
                tot += w * np.exp(-0.5 * ((z - mu) / sigma) ** 2) / (sigma * math.sqrt(2 * math.pi))
            else:
                a = (l[0] - 1.0 - H) if j < 0 else l[j] - H
                b = (l[0] + H) if j < 0 else l[j + 1] + H
                tot += w * np.where((z >= a) & (z < b), 1.0 / (b - a), 0.0)
        return tot

    def F_of_cell(k):
        # z inside cell k: cells before k were passed (empty), cell k stopped the beam (occupied),
        # cells after k are not informed (delta = 1, zero gain).
        s = 0.0
        for i in range(n):
            if i in skip:
                continue
            if i < k:
                s += _gain(delta_emp, o[i])
            elif i == k:
                s += _gain(delta_occ, o[i])
        return s

    xg, wg = np.polynomial.legendre.leggauss(order)
    total = 0.0
    for k in range(n):
        Fk = F_of_cell(k)
        if Fk == 0.0:
            continue
        a, b = l[k], l[k + 1]
        if noise == "uniform":
            # integrand is piecewise constant with breakpoints at the uniform supports' ends
            pts = sorted({a, b} | {v for w, j in comps for v in (
                ((l[0] - 1.0 - H) if j < 0 else l[j] - H), ((l[0] + H) if j < 0 else l[j + 1] + H)) if a < v < b})
            mass = 0.0
            for lo, hi in zip(pts[:-1], pts[1:]):
                mass += density(np.array([0.5 * (lo + hi)]))[0] * (hi - lo)
            total += Fk * mass
            continue
        edges = np.linspace(a, b, panels + 1)
        mass = 0.0
        for lo, hi in zip(edges[:-1], edges[1:]):
            z = 0.5 * (hi - lo) * xg + 0.5 * (hi + lo)
            mass += 0.5 * (hi - lo) * float(np.dot(wg, density(z)))
        total += Fk * mass
    return total


def exact_cells(W, H, ox, oy, dx, dy, R):
    """Cells of the grid [0,W)x[0,H) that the ray o + lam * d / 2^30 (o in Q16) crosses with
    positive length for lam in (0, R), in order, with their entry parameters (clamped at 0), and
    the end parameter min(R, grid exit). Exact rational arithmetic."""
    oxf, oyf = Fraction(ox, 1 << 16), Fraction(oy, 1 << 16)
    dxf, dyf = Fraction(dx, 1 << 30), Fraction(dy, 1 << 30)
    R = Fraction(R)

    def slab(o_, d_, lo, hi):
        if d_ == 0:
            return (None, None) if lo <= o_ <= hi else (1, 0)  # (None, None) = unbounded
        t1, t2 = (lo - o_) / d_, (hi - o_) / d_
        return (min(t1, t2), max(t1, t2))

    # grid exit
    gx = slab(oxf, dxf, 0, W)
    gy = slab(oyf, dyf, 0, H)
    ends = [v[1] for v in (gx, gy) if v[0] is not None]
    exit_lam = min(ends) if ends else R
    cells = []
    for cy in range(H):
        for cx in range(W):
            sx = slab(oxf, dxf, cx, cx + 1)
            sy = slab(oyf, dyf, cy, cy + 1)
            if (sx[0] is not None and sx[0] > sx[1]) or (sy[0] is not None and sy[0] > sy[1]):
                continue
            lo = max([v[0] for v in (sx, sy) if v[0] is not None] + [Fraction(0)])
            hi_c = [v[1] for v in (sx, sy) if v[0] is not None]
            hi = min(hi_c) if hi_c else R
            if hi > lo and lo < R and lo < exit_lam:
                # an axis-parallel ray along a shared grid line belongs to the cell above/right
                if dxf == 0 and oxf == cx + 1:
                    continue
                if dyf == 0 and oyf == cy + 1:
                    continue
                cells.append((lo, cy * W + cx))
    cells.sort()
    return [c for _, c in cells], [float(v) for v, _ in cells], float(min(R, exit_lam))
