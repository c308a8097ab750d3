"""Pins of the oracle's per-cell quantities (Section 2.2, Algorithms 2 and 3) against
definitions that do not pass through the oracle: the Bernoulli KL divergence, enumeration of all
2^n maps, and the piecewise-constant form of Lemma 1."""
import itertools
import math

import numpy as np
import pytest

from tests.bruteforce import kl_gain


@pytest.mark.parametrize("delta", [1.5, 0.67, 1 / 1.5, 3.0, 0.2])
def test_f_equals_bernoulli_kl(orc, delta):
    # f(delta, r) is the KL divergence between the cell's posterior (odds times delta) and prior.
    for o in np.linspace(0.01, 0.99, 41):
        ref = kl_gain(delta, o)
        assert orc.f_prob(delta, o) == pytest.approx(ref, rel=1e-12, abs=1e-15)
        assert orc.f_odds(delta, o / (1 - o)) == pytest.approx(ref, rel=1e-10, abs=1e-14)


def test_f_nonnegative_and_zero_on_known_cells(orc):
    for delta in (1.5, 0.67, 4.0, 0.1):
        assert orc.f_prob(delta, 0.0) == 0.0
        assert abs(orc.f_prob(delta, 1.0)) < 1e-15
        for o in np.linspace(0, 1, 101):
            assert orc.f_prob(delta, o) >= -1e-16
    for o in np.linspace(0, 1, 11):
        assert orc.f_prob(1.0, o) == 0.0  # delta = 1: no information (Lemma 1 proof)


def test_f_emp_is_f_occ_of_inverse_odds(orc):
    # Section 3.3: with delta_emp * delta_occ = 1, f(delta_emp, r) = f(delta_occ, 1/r).
    for r in (0.05, 0.3, 1.0, 2.5, 19.0):
        assert orc.f_odds(1 / 1.5, r) == pytest.approx(orc.f_odds(1.5, 1 / r), rel=1e-12)


def test_first_hit_matches_map_enumeration(orc):
    rng = np.random.default_rng(7)
    for n in (1, 2, 5, 9):
        o = rng.uniform(0, 1, n)
        pe = orc.first_hit(o)
        ref = np.zeros(n + 1)
        for m in itertools.product((0, 1), repeat=n):
            p = math.prod(o[i] if m[i] else 1 - o[i] for i in range(n))
            first = next((i + 1 for i in range(n) if m[i]), 0)
            ref[first] += p
        np.testing.assert_allclose(pe, ref, rtol=1e-12, atol=1e-15)
        assert pe.sum() == pytest.approx(1.0, abs=1e-12)


def test_c_k_is_lemma1_piecewise_sum(orc):
    # Lemma 1: for z in cell k, F(z) = sum_i f(delta_i(z), r_i) with delta_emp before k,
    # delta_occ at k and 1 after k.
    rng = np.random.default_rng(3)
    o = rng.uniform(0.01, 0.99, 12)
    C = orc.c_k(o, 1.5, 0.67)
    for k in range(12):
        F = sum(kl_gain(0.67, o[i]) for i in range(k)) + kl_gain(1.5, o[k])
        assert C[k] == pytest.approx(F, rel=1e-12)
