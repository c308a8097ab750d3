"""Index arithmetic of the exact 2D kernel's window (csrc/eval2d.cuh exact_pairs_sum), replayed on
the CPU in FP32 over whole beams: the pair counts found by the coverage trials are the fewest that
cover every slot of a round, every boundary within the cut of a slot's centre lies in the pairs
that slot visits, the trials end, and every pair read stays inside the padded pair array (16
padding pairs on each side). The replay follows the kernel step by step (rounds of 64 slots, two
adjacent slots per lane, while more than 32 remain, then rounds of 32 slots, one per lane; trials
starting from the previous round's counts); the GPU tests check the sums themselves."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_1905_02238_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
F = np.float32


def _consts():
    src = open(os.path.join(ROOT, "paper_1905_02238_gb300", "csrc", "eval2d.cuh")).read()
    cuts = dict(re.findall(r"constexpr float (kTailCut\w*) = ([0-9.]+)f;", src))
    pad = int(re.search(r"constexpr int kPad2D = (\d+);", src).group(1))
    return F(cuts["kTailCutDefault"]), F(cuts["kTailCut"]), pad


def _trials(G, side, ok, n):
    g, steps = G[side], 0
    if ok(g):
        while g > 0 and ok(g - 1):
            g -= 1
    else:
        while not ok(g):
            g += 1
            steps += 1
            assert steps <= n + 2, "trials do not end"
    assert g == 0 or not ok(g - 1)  # the fewest pairs that cover the round
    G[side] = g


def _covered(sl, n, lo, hi, mu, cut):
    b, c = F(mu - cut), F(mu + cut)
    for k in range(n + 1):
        if b <= sl[k] < c:  # within the cut of the centre, in the kernel's FP32 comparisons
            assert lo <= k < hi, (k, lo, hi)


def replay(sl, e0, cut, pad, cs):
    """sl: float32 scaled boundaries l_0..l_n of one beam; cs: scaled length of one cell."""
    n = len(sl) - 1
    nslots = n + (1 if e0 else 0)
    get = lambda i: sl[i] if 0 <= i <= n else (F(-3e30) if i < 0 else F(3e30))  # padded pairs
    span = sl[n] - sl[0]
    per = F(n) / span if span > F(0) else F(0)
    G = {"neg": int(min(cut * per, F(n + 1))) >> 1}
    G["pos"] = G["neg"]
    mtop = ((n >> 1) + 1 + pad // 2) * 2  # pairs (m, m + 1) read stay below this m
    mu0 = F(sl[0] - F(0.5) * F(cs))  # the no-return slot's centre, l_1 - 1/2 (scaled)
    jb = 0
    while n - jb > 32:  # two adjacent slots per lane
        j = jb + 2 * np.arange(32)
        actA, actB = j < n, j + 1 < n
        a = np.where(actA, j, jb)
        muA = np.array([F(F(0.5) * (get(k) + get(k + 1))) for k in a], dtype=F)
        muB = np.array([F(F(0.5) * (get(k + 1) + get(k + 2))) for k in a], dtype=F)
        below = (muA - cut).astype(F)
        above = (np.where(actB, muB, muA) + cut).astype(F)
        _trials(G, "neg", lambda g: all((not x) or m <= 0 or get(m - 1) < b
                                        for x, m, b in zip(actA, a - 2 * g, below)), n)
        _trials(G, "pos", lambda g: all((not x) or e > n or get(e) >= c
                                        for x, e, c in zip(actA, a + 2 + 2 * g, above)), n)
        for x, y, aa, ma, mb in zip(actA, actB, a, muA, muB):
            lo = max(aa - 2 * G["neg"], -pad)
            hi = min(aa + 2 + 2 * G["pos"], mtop)
            assert lo % 2 == 0 and hi % 2 == 0 and lo <= aa < hi
            assert lo >= -pad and hi <= mtop
            assert aa + 2 <= mtop - 1  # the centre of B reads l_{a+2} inside the pairs
            if x:
                _covered(sl, n, lo, hi, ma, cut)
            if y:
                _covered(sl, n, lo, hi, mb, cut)
        jb += 64
    while jb < nslots:  # one slot per lane (and the no-return slot)
        j = np.arange(jb, jb + 32)
        act = j < nslots
        cell = act & (j < n)
        mid = np.where(cell, j + 1, 0)
        mu = np.array([F(F(0.5) * (sl[k] + sl[k + 1])) if c else (mu0 if x else F(0))
                       for k, c, x in zip(j, cell, act)], dtype=F)
        nb = mid & ~1
        below, above = (mu - cut).astype(F), (mu + cut).astype(F)
        _trials(G, "neg", lambda g: all((not x) or m <= 0 or get(m - 1) < b for x, m, b in zip(act, nb - 2 * g, below)),
                n)
        _trials(G, "pos", lambda g: all((not x) or e > n or get(e) >= c for x, e, c in zip(act, nb + 2 + 2 * g, above)),
                n)
        for x, m, u in zip(act, nb, mu):
            if not x:
                continue
            lo = max(m - 2 * G["neg"], -pad)
            hi = min(m + 2 + 2 * G["pos"], mtop)
            assert lo % 2 == 0 and hi % 2 == 0 and lo <= m < hi
            assert lo >= -pad and hi <= mtop
            _covered(sl, n, lo, hi, u, cut)
        jb += 32


@pytest.mark.parametrize("sigma", [0.5, 2.0, 12.0])
@pytest.mark.parametrize("e0", [0, 1])
def test_window_on_traversed_beams(sigma, e0):
    cut, full, pad = _consts()
    grid, poses, dirs = synth.random_grid_200()
    H, W = grid.shape
    cs = np.sqrt(np.log2(np.e)) / (sigma * np.sqrt(2.0))
    for b in range(0, dirs.shape[0], 23):
        d = oracle.beam_dir_2d(poses[0], dirs[b])
        _, l = oracle.trace_2d(W, H, poses[0][0], poses[0][1], d[0], d[1], 64.0)
        if len(l) < 2:
            continue
        sl = (l * cs).astype(F)
        for c in (cut, full):
            replay(sl, e0, c, pad, cs)


@pytest.mark.parametrize("e0", [0, 1])
def test_window_on_explicit_beams(e0):
    # zero-length cells, long cells, and boundaries denser than any traversal
    cut, full, pad = _consts()
    for seed, (wlo, whi) in enumerate(((0.0, 0.3), (0.05, 1.4142), (20.0, 60.0))):
        off, _, l, lend = synth.random_beams(12, 1, 300, seed=80 + seed, w_lo=wlo, w_hi=whi)
        for b in range(12):
            edges = np.concatenate([l[off[b]:off[b + 1]], [lend[b]]]).astype(np.float64)
            for sigma in (0.5, 3.0):
                cs = np.sqrt(np.log2(np.e)) / (sigma * np.sqrt(2.0))
                sl = (edges * cs).astype(F)
                for c in (cut, full):
                    replay(sl, e0, c, pad, cs)
