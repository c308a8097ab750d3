"""Index arithmetic of the exact 2D kernel's window (csrc/eval2d.cuh exact_window_sum), replayed on
the CPU in FP32 over whole beams: the pair counts found by the coverage trials are the fewest that
cover every slot of a round, every boundary within the cut of a slot's centre lies in the pairs
that slot visits, the trials end, and every pair read stays inside the padded arrays (32 padding
boundaries on each side). The replay follows the kernel step by step (rounds of 32 slots, trials
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


def replay(sl, e0, cut, pad, cs):
    """sl: float32 scaled boundaries l_0..l_n of one beam; cs: scaled length of one cell."""
    n = len(sl) - 1
    nslots = n + (1 if e0 else 0)
    get = lambda i: sl[i] if 0 <= i <= n else (F(-3e30) if i < 0 else F(3e30))  # padded array
    span = sl[n] - sl[0]
    per = F(n) / span if span > F(0) else F(0)
    G = {"neg": int(min(cut * per, F(n + 1))) >> 1}
    G["pos"] = G["neg"]
    mtop = (n + 1 + pad) & ~1
    mu0 = sl[0] - F(0.5) * F(cs)  # the no-return slot's centre, l_1 - 1/2
    for jb in range(0, nslots, 32):
        j = np.arange(jb, jb + 32)
        act = j < nslots
        cell = act & (j < n)
        mid = np.where(cell, j + 1, 0)
        mu = np.array([F(0.5) * (sl[k] + sl[k + 1]) if c else (mu0 if a else F(0)) for k, c, a in zip(j, cell, act)],
                      dtype=F)
        nb = mid & ~1
        below, above = (mu - cut).astype(F), (mu + cut).astype(F)
        ok = {
            "neg": lambda g: all((not a) or m <= 0 or get(m - 1) < b for a, m, b in zip(act, nb - 2 * g, below)),
            "pos": lambda g: all((not a) or e > n or get(e) >= b for a, e, b in zip(act, nb + 2 + 2 * g, above)),
        }
        for side in ("neg", "pos"):
            g, steps = G[side], 0
            if ok[side](g):
                while g > 0 and ok[side](g - 1):
                    g -= 1
            else:
                while not ok[side](g):
                    g += 1
                    steps += 1
                    assert steps <= n + 2, "trials do not end"
            assert g == 0 or not ok[side](g - 1)  # the fewest pairs that cover the round
            G[side] = g
        m0 = np.where(act, np.maximum(nb - 2 * G["neg"], -pad), 0)
        end = np.where(act, np.minimum(nb + 2 + 2 * G["pos"], mtop), 0)
        for a, lo, hi, b, c, m in zip(act, m0, end, below, above, nb):
            if not a:
                continue
            assert lo % 2 == 0 and hi % 2 == 0 and lo <= m < hi
            assert lo >= -pad and hi - 1 <= n + pad  # pairs (m, m + 1) read inside the padding
            for k in range(n + 1):
                if b <= sl[k] < c:  # within the cut of the centre, in the kernel's FP32 comparisons
                    assert lo <= k < hi, (k, lo, hi)


@pytest.mark.parametrize("sigma", [0.5, 2.0, 12.0])
@pytest.mark.parametrize("e0", [0, 1])
def test_window_on_traversed_beams(sigma, e0):
    cut, full, pad = _consts()
    grid, poses, dirs = synth.config1()
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
