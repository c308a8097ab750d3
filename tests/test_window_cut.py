"""The exact 2D kernel's window (csrc/eval2d.cuh) skips only what FP32 cannot resolve: the
default cut leaves every skipped boundary term below 2^-27 of its weight and the skipped terms
of one side of a cell centre at most 2^-24 (one FP32 ulp) of the largest weight |C_m - C_{m-1}|
for sigma up to 19 cells, below 2^-25 for sigma <= 2, on traversed beams (at most two boundaries
per major-axis crossing); beyond the full-window cut the factor 2^(-s^2) is subnormal, so
ex2.approx.ftz returns 0. Checked in FP64 on the CPU from the paper's Gaussian tail (Theorem 1's
G as a Phi difference)."""
import os
import re

import numpy as np
import pytest
from scipy.special import erfc

import oracle
from paper_1905_02238_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SQ = np.sqrt(np.log2(np.e))  # scaled distance s = x sqrt(log2 e) / (sigma sqrt 2): exp(-z^2) = 2^(-s^2)


def _cuts():
    src = open(os.path.join(ROOT, "paper_1905_02238_gb300", "csrc", "eval2d.cuh")).read()
    vals = dict(re.findall(r"constexpr float (kTailCut\w*) = ([0-9.]+)f;", src))
    return float(vals["kTailCutDefault"]), float(vals["kTailCut"])


def _tail(s):
    return 0.5 * erfc(np.abs(s) / SQ)  # upper Gaussian tail at scaled distance s


def test_cut_constants():
    cut, full = _cuts()
    assert _tail(cut) < 2.0 ** -27
    assert full * full > 126.0  # 2^(-s^2) below the smallest normal FP32 beyond the full window
    for sigma in (0.5, 1.0, 2.0, 5.0, 10.0, 19.0, 20.0):
        cs = SQ / (sigma * np.sqrt(2.0))  # scaled length of one cell
        # two boundaries per crossing interval at most; successive intervals shrink the tail by
        # 2^(-2 cut cs) at least: the geometric bound of one side
        bound = 2.0 * _tail(cut) / (1.0 - 2.0 ** (-2.0 * cut * cs))
        assert bound <= 2.0 ** -24 * (1.0 if sigma <= 19.0 else 1.01)
        if sigma <= 2.0:
            assert bound < 2.0 ** -25


@pytest.mark.parametrize("sigma", [0.7, 2.0, 20.0])
def test_skipped_terms_on_traversed_beams(sigma):
    cut, _ = _cuts()
    grid, poses, dirs = synth.random_grid_200()
    H, W = grid.shape
    cs = SQ / (sigma * np.sqrt(2.0))
    worst = 0.0
    for b in range(0, dirs.shape[0], 9):
        d = oracle.beam_dir_2d(poses[0], dirs[b])
        cells, l = oracle.trace_2d(W, H, poses[0][0], poses[0][1], d[0], d[1], 64.0)
        n = len(cells)
        if n == 0:
            continue
        o = grid.reshape(-1)[cells].astype(np.float64)
        C = np.concatenate([[0.0], oracle.c_k(o, 1.5, 0.67), [0.0]])
        dC = np.abs(C[1:] - C[:-1])  # weights of boundaries 0..n
        ls = l * cs
        mu = 0.5 * (ls[:-1] + ls[1:])
        for j in range(n):
            dist = ls - mu[j]
            for side in (dist < 0, dist >= 0):
                skip = side & (np.abs(dist) >= cut)
                if not skip.any():
                    continue
                mass = np.sum(dC[skip] * _tail(dist[skip]))
                worst = max(worst, mass / max(dC.max(), 1e-300))
                assert np.all(_tail(dist[skip]) < 2.0 ** -27)
    assert worst <= 2.0 ** -24
