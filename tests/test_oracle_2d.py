"""Pins of the oracle's 2D variants (Theorem 1 / Algorithm 1, eq. fsmi_approx, Theorem 4 /
Algorithm 4) against brute-force numerical integration of the mutual-information definition
(eq. mi_sum), closed forms and limits that the paper's derivations fix."""
import math

import numpy as np
import pytest

from tests.bruteforce import smi_integral


def _beam(rng, n, unit=False, lo=0.0, hi=1.0):
    o = rng.uniform(lo, hi, n)
    w = np.ones(n) if unit else rng.uniform(0.1, 1.4, n)
    l = np.concatenate([[0.0], np.cumsum(w)])
    return o, l


@pytest.mark.parametrize("sigma", [0.3, 0.7, 1.5])
@pytest.mark.parametrize("e0", [0, 1])
def test_fsmi_matches_numerical_integral(orc, sigma, e0):
    # Theorem 1 against the SMI-style integral of the definition (Section 2.2).
    rng = np.random.default_rng(int(sigma * 10) + 100 * e0)
    for n in (1, 3, 7, 12):
        o, l = _beam(rng, n)
        prm = orc.Params(variant=orc.EXACT, sigma=sigma, delta_occ=1.5, delta_emp=0.67, e0_mode=e0)
        got = orc.fsmi_beam(o, l, prm)
        ref = smi_integral(o, l, sigma, 1.5, 0.67, e0_mode=e0)
        assert got == pytest.approx(ref, rel=1e-9, abs=1e-13)


@pytest.mark.parametrize("H", [1, 2, 4])
@pytest.mark.parametrize("e0", [0, 1])
def test_uniform_three_ways(orc, H, e0):
    # Theorem 4: the D-prefix formula of Algorithm 4 = the generic pair sum with the uniform
    # density = the integral of the definition with P(z|e_j) = U[l_j - H, l_{j+1} + H].
    rng = np.random.default_rng(H + 10 * e0)
    for n in (1, 2, 5, 11):
        o, l = _beam(rng, n, unit=True)
        prm = orc.Params(variant=orc.UNIFORM, uniform_h=H, delta_occ=1.5, delta_emp=0.67, e0_mode=e0)
        a = orc.fsmi_beam(o, l, prm)
        b = orc.uniform_pairsum(o, l, prm)
        c = smi_integral(o, l, 1.0, 1.5, 0.67, e0_mode=e0, noise="uniform", H=H)
        assert a == pytest.approx(b, rel=1e-12, abs=1e-15)
        assert a == pytest.approx(c, rel=1e-12, abs=1e-15)


def test_mi_zero_on_known_map(orc):
    rng = np.random.default_rng(5)
    for variant in (orc.EXACT, orc.APPROX, orc.UNIFORM):
        for _ in range(5):
            n = int(rng.integers(1, 30))
            o = rng.integers(0, 2, n).astype(float)
            l = np.concatenate([[0.0], np.cumsum(rng.uniform(0.2, 1.4, n))])
            prm = orc.Params(variant=variant, sigma=1.0, trunc_delta=2, uniform_h=2)
            assert abs(orc.fsmi_beam(o, l, prm)) < 1e-15


def test_mi_nonnegative(orc):
    rng = np.random.default_rng(6)
    for variant in (orc.EXACT, orc.APPROX, orc.UNIFORM):
        for _ in range(20):
            o, l = _beam(rng, int(rng.integers(1, 40)))
            prm = orc.Params(variant=variant, sigma=float(rng.uniform(0.2, 3)), trunc_delta=3, uniform_h=2,
                             e0_mode=int(rng.integers(0, 2)))
            assert orc.fsmi_beam(o, l, prm) >= 0.0


def test_single_cell_closed_form(orc):
    # n = 1: I = o * f(delta_occ, r) * (2 Phi(w / (2 sigma)) - 1).
    for o in (0.1, 0.5, 0.9):
        for w in (0.3, 1.0, 1.4):
            for sigma in (0.2, 1.0, 2.5):
                prm = orc.Params(sigma=sigma)
                ref = o * orc.f_prob(1.5, o) * math.erf(w / (2 * sigma * math.sqrt(2)))
                assert orc.fsmi_beam([o], [0.0, w], prm) == pytest.approx(ref, rel=1e-13)


def test_small_sigma_limit(orc):
    # sigma -> 0: G_{k,j} -> 1[k = j], so I -> sum_j P(e_j) C_j.
    rng = np.random.default_rng(8)
    o, l = _beam(rng, 25)
    pe = orc.first_hit(o)
    C = orc.c_k(o, 1.5, 0.67)
    ref = float(np.dot(pe[1:], C))
    assert orc.fsmi_beam(o, l, orc.Params(sigma=1e-4)) == pytest.approx(ref, rel=1e-12)


def test_approx_limits(orc):
    rng = np.random.default_rng(9)
    for _ in range(5):
        n = int(rng.integers(2, 40))
        o, l = _beam(rng, n)
        sigma = float(rng.uniform(0.3, 3.0))
        for e0 in (0, 1):
            ex = orc.fsmi_beam(o, l, orc.Params(variant=orc.EXACT, sigma=sigma, e0_mode=e0))
            # Delta >= n keeps every pair: Approx-FSMI = FSMI
            ap = orc.fsmi_beam(o, l, orc.Params(variant=orc.APPROX, sigma=sigma, trunc_delta=n, e0_mode=e0))
            assert ap == pytest.approx(ex, rel=1e-14)
            # nondecreasing in Delta (all terms are >= 0)
            vals = [orc.fsmi_beam(o, l, orc.Params(variant=orc.APPROX, sigma=sigma, trunc_delta=d, e0_mode=e0))
                    for d in range(0, n + 1)]
            assert all(b >= a - 1e-15 for a, b in zip(vals, vals[1:]))
        # Delta = 0 keeps only G_{j,j} = erf(w_j / (2 sqrt(2) sigma))
        pe = orc.first_hit(o)
        C = orc.c_k(o, 1.5, 0.67)
        w = np.diff(l)
        ref = sum(pe[j + 1] * C[j] * math.erf(w[j] / (2 * math.sqrt(2) * sigma)) for j in range(n))
        d0 = orc.fsmi_beam(o, l, orc.Params(variant=orc.APPROX, sigma=sigma, trunc_delta=0))
        assert d0 == pytest.approx(ref, rel=1e-13)


def test_uniform_h_remark(orc):
    # Remark after Theorem 4: H = round(sqrt(3) sigma - 1/2) matches the Gaussian's variance;
    # with that H the uniform result stays close to the exact one on a long random beam.
    rng = np.random.default_rng(10)
    o, l = _beam(rng, 80, unit=True, lo=0.05, hi=0.5)
    sigma = 3.0
    H = int(round(math.sqrt(3) * sigma - 0.5))
    ex = orc.fsmi_beam(o, l, orc.Params(variant=orc.EXACT, sigma=sigma))
    un = orc.fsmi_beam(o, l, orc.Params(variant=orc.UNIFORM, uniform_h=H))
    assert un == pytest.approx(ex, rel=0.1)
