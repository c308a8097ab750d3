"""Pins of the oracle's 3D/RLE path (Section 4): virtual-cell sampling, run-length encoding
(eq. occup_rle), and the three RLE variants (Theorems 3, 5, 6) against the cell-level sums they
are derived from, the A/B identities of Theorem 3, Lemma 6 and the 2D variants."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1905_02238_gb300 import synth


# ---- sampling and encoding --------------------------------------------------------------------

def test_sample_3d_matches_exact_positions(orc):
    rng = np.random.default_rng(21)
    X, Y, Z = 11, 9, 7
    vox = rng.uniform(0, 1, (Z, Y, X)).astype(np.float32)
    dirs = synth.pinhole_dirs(4, 4, 120.0)
    for _ in range(20):
        pose = synth.pose_3d(*rng.uniform([0, 0, 0], [X, Y, Z]), yaw=rng.uniform(0, 6.3), pitch=rng.uniform(-1, 1))
        u = dirs[int(rng.integers(0, len(dirs)))]
        got = orc.sample_3d(vox, pose, u, 30)
        # the rotated direction, rounded half up, then the voxel holding o + (i + 1/2) d exactly
        d = [((sum(int(pose[3 + 3 * r + c]) * int(u[c]) for c in range(3)) + (1 << 29)) >> 30) for r in range(3)]
        ref = []
        for i in range(30):
            p = [Fraction(int(pose[a]), 1 << 16) + Fraction(2 * i + 1, 2) * Fraction(d[a], 1 << 30) for a in range(3)]
            v = [math.floor(c) for c in p]
            if not (0 <= v[0] < X and 0 <= v[1] < Y and 0 <= v[2] < Z):
                break
            ref.append(vox[v[2], v[1], v[0]])
        np.testing.assert_array_equal(got, np.array(ref, np.float32))


def test_rle_roundtrip_maximal_and_capped(orc):
    rng = np.random.default_rng(22)
    for cap in (1, 3, 64):
        for _ in range(30):
            n = int(rng.integers(0, 300))
            vals = rng.choice(np.array([0.1, 0.5, 0.9, 0.3], np.float32), size=n, p=[0.6, 0.2, 0.1, 0.1])
            rep = rng.integers(1, 40, size=n)
            s = np.repeat(vals, rep)[:n]
            ro, rl = orc.rle_encode(s, cap)
            np.testing.assert_array_equal(np.repeat(ro, rl), s)
            assert np.all(rl >= 1) and np.all(rl <= cap)
            for u in range(1, len(ro)):  # adjacent runs differ, or the previous one is full
                assert ro[u] != ro[u - 1] or rl[u - 1] == cap


# ---- cell-level references ----------------------------------------------------------------------

def _cells(ro, rl):
    return np.repeat(np.asarray(ro, np.float64), np.asarray(rl))


def _pe_c(orc, o, docc=1.5, demp=0.67):
    o = np.asarray(o, np.float64)
    surv = np.concatenate([[1.0], np.cumprod(1 - o)])
    pe = surv[:-1] * o
    fo = np.array([orc.f_prob(docc, v) for v in o])
    fe = np.array([orc.f_prob(demp, v) for v in o])
    C = np.concatenate([[0.0], np.cumsum(fe)])[:-1] + fo
    return pe, C


def _cell_pair_sum(pe, C, g):
    n = len(pe)
    idx = np.arange(n)
    G = g(idx[None, :] - idx[:, None])  # G[j, k] = g(k - j)
    return float(pe @ G @ C)


def test_theorem3_expansion_pdf(orc):
    # eq. (eqn_from_fsmi): FSMI-RLE(runs) = sum_j sum_k P(e_j) C_k G_{k,j} over the virtual cells,
    # with G the point density of eq. (p_e_u)-(C_v).
    rng = np.random.default_rng(23)
    for sigma in (0.6, 2.0):
        for _ in range(6):
            nr = int(rng.integers(1, 9))
            ro = rng.uniform(0.02, 0.98, nr).astype(np.float32)
            rl = rng.integers(1, 9, nr)
            pe, C = _pe_c(orc, _cells(ro, rl))
            ref = _cell_pair_sum(pe, C, lambda d: np.exp(-d * d / (2 * sigma * sigma)) / (math.sqrt(2 * math.pi) * sigma))
            got = orc.rle_beam(ro, rl, orc.Params(variant=orc.EXACT, sigma=sigma, g_kernel=orc.G_PDF))
            assert got == pytest.approx(ref, rel=1e-12)


def test_erf_kernel_equals_2d_fsmi_on_unit_cells(orc):
    # with the cell-integrated kernel, FSMI-RLE on runs = FSMI (Theorem 1) on the decompressed
    # unit cells (which test_oracle_2d pins to the integral of the definition).
    rng = np.random.default_rng(24)
    for _ in range(8):
        nr = int(rng.integers(1, 10))
        ro = rng.uniform(0.02, 0.98, nr).astype(np.float32)
        rl = rng.integers(1, 7, nr)
        o = _cells(ro, rl)
        l = np.arange(len(o) + 1, dtype=np.float64)
        sigma = float(rng.uniform(0.4, 3.0))
        a = orc.rle_beam(ro, rl, orc.Params(variant=orc.EXACT, sigma=sigma, g_kernel=orc.G_ERF))
        b = orc.fsmi_beam(o, l, orc.Params(variant=orc.EXACT, sigma=sigma))
        assert a == pytest.approx(b, rel=1e-12)


def test_uniform_rle_equals_uniform_fsmi(orc):
    # Theorem 6 (with Theorem 3's algebra) = Algorithm 4 on the decompressed unit cells.
    rng = np.random.default_rng(25)
    for H in (1, 2, 4):
        for _ in range(6):
            nr = int(rng.integers(1, 10))
            ro = rng.uniform(0.02, 0.98, nr).astype(np.float32)
            rl = rng.integers(1, 9, nr)
            o = _cells(ro, rl)
            l = np.arange(len(o) + 1, dtype=np.float64)
            a = orc.rle_beam(ro, rl, orc.Params(variant=orc.UNIFORM, uniform_h=H))
            b = orc.fsmi_beam(o, l, orc.Params(variant=orc.UNIFORM, uniform_h=H))
            assert a == pytest.approx(b, rel=1e-12)


def test_approx_rle_readings_sandwich(orc):
    # all terms are >= 0: strict band <= Theorem 5 sub-blocks <= FSMI-RLE, equal at Delta >= n;
    # the strict band equals the cell-level band sum.
    rng = np.random.default_rng(26)
    sigma = 2.0
    g = lambda d: np.exp(-d * d / (2 * sigma * sigma)) / (math.sqrt(2 * math.pi) * sigma)
    for _ in range(10):
        nr = int(rng.integers(1, 10))
        ro = rng.uniform(0.02, 0.98, nr).astype(np.float32)
        rl = rng.integers(1, 12, nr)
        n = int(rl.sum())
        for D in (0, 1, 3, 6, n):
            full = orc.rle_beam(ro, rl, orc.Params(variant=orc.EXACT, sigma=sigma))
            thm = orc.rle_beam(ro, rl, orc.Params(variant=orc.APPROX, sigma=sigma, trunc_delta=D, approx_reading=0))
            band = orc.rle_beam(ro, rl, orc.Params(variant=orc.APPROX, sigma=sigma, trunc_delta=D, approx_reading=1))
            pe, C = _pe_c(orc, _cells(ro, rl))
            ref_band = _cell_pair_sum(pe, C, lambda d: np.where(np.abs(d) <= D, g(d), 0.0))
            assert band == pytest.approx(ref_band, rel=1e-12, abs=1e-300)
            assert band <= thm * (1 + 1e-12) + 1e-300
            assert thm <= full * (1 + 1e-12)
            if D >= n:
                assert thm == pytest.approx(full, rel=1e-12)
                assert band == pytest.approx(full, rel=1e-12)


def test_theorem5_sub_blocks_keep_all_band_pairs(orc):
    # Theorem 5 as printed equals the cell-level pair sum restricted to the diagonal blocks and
    # the sub-blocks [s_u', s_u' + L_u') x [s_v', s_v' + L_v') of eqs. (su')-(Lv'): this pins the
    # run-level weights P_E(u)(1 - o_u)^(s_u' - s_u) and D_E(v) + (s_v' - s_v) f_emp(v).
    rng = np.random.default_rng(27)
    sigma = 1.5
    for _ in range(10):
        nr = int(rng.integers(2, 8))
        ro = rng.uniform(0.02, 0.98, nr).astype(np.float32)
        rl = rng.integers(1, 10, nr)
        D = int(rng.integers(1, 5))
        s = np.concatenate([[0], np.cumsum(rl)])
        run_of = np.repeat(np.arange(nr), rl)
        n = int(s[-1])
        keep = np.zeros((n, n), bool)
        for j in range(n):
            for k in range(n):
                u, v = run_of[j], run_of[k]
                if u == v:
                    keep[j, k] = True
                elif u < v:
                    keep[j, k] = s[v] < s[u] + rl[u] + D and j >= max(s[u], s[v] - D) and k < s[v] + min(rl[v], s[u] + rl[u] + D - s[v])
                else:
                    keep[j, k] = s[u] < s[v] + rl[v] + D and j < s[u] + min(rl[u], s[v] + rl[v] + D - s[u]) and k >= max(s[v], s[u] - D)
        pe, C = _pe_c(orc, _cells(ro, rl))
        idx = np.arange(n)
        G = np.exp(-(idx[None, :] - idx[:, None]) ** 2 / (2 * sigma * sigma)) / (math.sqrt(2 * math.pi) * sigma)
        ref = float(pe @ (G * keep) @ C)
        got = orc.rle_beam(ro, rl, orc.Params(variant=orc.APPROX, sigma=sigma, trunc_delta=D, approx_reading=0))
        assert got == pytest.approx(ref, rel=1e-12)


def test_theorem5_equals_contiguous_cell_windows(orc):
    # The form the CUDA path evaluates: for a first-hit cell j of run u, Theorem 5 keeps exactly the
    # cells [lo_j, hi_j) with lo_j = max(s of the run holding j - Delta, s_u - Delta) and
    # hi_j = min(e_u + Delta, e of the run holding j + Delta) (clamped to the ray; e one past a
    # run's last cell). Checked against the oracle's Theorem 5 (pinned above to its sub-block mask)
    # on random runs, Delta from 0 up to past the ray's length.
    rng = np.random.default_rng(31)
    sigma = 1.5
    for _ in range(40):
        nr = int(rng.integers(1, 9))
        ro = rng.uniform(0.02, 0.98, nr).astype(np.float32)
        rl = rng.integers(1, 12, nr)
        D = int(rng.integers(0, 14))
        s = np.concatenate([[0], np.cumsum(rl)])
        run_of = np.repeat(np.arange(nr), rl)
        n = int(s[-1])
        pe, C = _pe_c(orc, _cells(ro, rl))
        ref = 0.0
        for j in range(n):
            u = run_of[j]
            lo = max(s[run_of[max(j - D, 0)]], s[u] - D)
            hi = min(s[u + 1] + D, s[run_of[min(j + D, n - 1)] + 1])
            k = np.arange(lo, hi)
            g = np.exp(-(k - j) ** 2 / (2 * sigma * sigma)) / (math.sqrt(2 * math.pi) * sigma)
            ref += pe[j] * float(g @ C[lo:hi])
        got = orc.rle_beam(ro, rl, orc.Params(variant=orc.APPROX, sigma=sigma, trunc_delta=D, approx_reading=0))
        assert got == pytest.approx(ref, rel=1e-12)


# ---- A and B (Theorem 3) ---------------------------------------------------------------------------

def _alpha(x, Lu, Lv, sigma, weight_k=False):
    s = 0.0
    for j in range(Lu):
        for k in range(Lv):
            s += (k if weight_k else 1) * x ** j * math.exp(-(j - k) ** 2 / (2 * sigma * sigma))
    return s


def test_A_B_shift_identities(orc):
    # eqs. (compute_A), (compute_B): A, B from alpha, beta by the t-shift.
    rng = np.random.default_rng(28)
    for _ in range(40):
        x = float(rng.uniform(0.05, 0.99))
        Lu, Lv = int(rng.integers(1, 7)), int(rng.integers(1, 7))
        t = int(rng.integers(-8, 9))
        sigma = float(rng.uniform(0.5, 3.0))
        A = orc.rle_A(0, sigma, 0, -1, x, Lu, Lv, t)
        B = orc.rle_B(0, sigma, 0, -1, x, Lu, Lv, t)
        if t >= 1:
            Aref = x ** (-t) * (_alpha(x, Lu + t, Lv, sigma) - _alpha(x, t, Lv, sigma))
            Bref = x ** (-t) * (_alpha(x, Lu + t, Lv, sigma, True) - _alpha(x, t, Lv, sigma, True))
        elif t == 0:
            Aref = _alpha(x, Lu, Lv, sigma)
            Bref = _alpha(x, Lu, Lv, sigma, True)
        else:
            Aref = _alpha(x, Lu, Lv - t, sigma) - _alpha(x, Lu, -t, sigma)
            Bref = _alpha(x, Lu, Lv - t, sigma, True) - _alpha(x, Lu, -t, sigma, True) + t * Aref
        assert A == pytest.approx(Aref, rel=1e-9, abs=1e-12)
        assert B == pytest.approx(Bref, rel=1e-9, abs=1e-12)


def test_lemma6_zero_pattern(orc):
    # Lemma 6: with G = 0 beyond Delta, A != 0 iff the two runs come within Delta of each other.
    rng = np.random.default_rng(29)
    for _ in range(200):
        D = int(rng.integers(0, 5))
        Lu, Lv = int(rng.integers(1, 6)), int(rng.integers(1, 6))
        if rng.random() < 0.5:  # u before v: s_v >= s_u + L_u, t = s_u - s_v <= -L_u
            t = -int(rng.integers(Lu, Lu + 8))
            nonzero = (-t) < Lu + D
        else:  # v before u: t = s_u - s_v >= L_v
            t = int(rng.integers(Lv, Lv + 8))
            nonzero = t < Lv + D
        A = orc.rle_A(0, 1.0, 0, D, 0.5, Lu, Lv, t)
        B = orc.rle_B(0, 1.0, 0, D, 0.5, Lu, Lv, t)
        assert (A != 0.0) == nonzero
        # B weights column k by k, so it also vanishes when only the k = 0 column is in reach;
        # what holds for B is: A = 0 implies B = 0.
        if not nonzero:
            assert B == 0.0


def test_rle_mi_zero_and_nonnegative(orc):
    rng = np.random.default_rng(30)
    for variant in (orc.EXACT, orc.APPROX, orc.UNIFORM):
        ro = rng.integers(0, 2, 6).astype(np.float32)
        rl = rng.integers(1, 9, 6)
        prm = orc.Params(variant=variant, sigma=2.0, trunc_delta=3, uniform_h=2)
        assert abs(orc.rle_beam(ro, rl, prm)) < 1e-15
        ro = rng.uniform(0, 1, 6).astype(np.float32)
        assert orc.rle_beam(ro, rl, prm) > 0.0


def test_e5_all_unit_runs_equal_cell_level(orc):
    # Section 5.4 shape with L = 1: FSMI-RLE on n single-cell runs is the cell-level pair sum.
    off, ro, rl = synth.e5_runs(1, nbeams=2, n=40)
    sigma = 2.0
    for b in range(2):
        r = ro[off[b]:off[b + 1]]
        pe, C = _pe_c(orc, r)
        ref = _cell_pair_sum(pe, C, lambda d: np.exp(-d * d / (2 * sigma * sigma)) / (math.sqrt(2 * math.pi) * sigma))
        assert orc.rle_beam(r, rl[off[b]:off[b + 1]], orc.Params(sigma=sigma)) == pytest.approx(ref, rel=1e-12)
