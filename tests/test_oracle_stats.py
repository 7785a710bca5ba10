"""Pins of the oracle's map statistics (Sect. 3.1, Eq. deltam) on hand-checkable cases."""
import math

import numpy as np
import pytest

from oracle import stats


def test_delta_m_definition_points():
    # mu = 1 -> 0 mag; mu = 10 -> -2.5 mag; mu = 100 -> -5 mag; empty -> +inf
    dm = stats.delta_m([100, 1000, 10000, 0], 100.0)
    assert dm[0] == 0.0 and dm[1] == pytest.approx(-2.5) and dm[2] == pytest.approx(-5.0)
    assert math.isinf(dm[3]) and dm[3] > 0


def test_rms_of_a_uniform_factor_is_its_magnitude():
    a = np.full(64, 200)
    b = np.full(64, 100)                      # every pixel twice as bright in a: 2.5 log10 2 mag
    r = stats.compare(a, 100.0, b, 100.0)
    assert r["rms_dm"] == pytest.approx(2.5 * math.log10(2.0), rel=1e-14)
    assert r["n_rms"] == 64 and r["zero_a"] == 0
    # N_rays rescales mu: the same counts with twice the rays per pixel are half as bright
    r2 = stats.compare(a, 200.0, b, 100.0)
    assert r2["rms_dm"] == pytest.approx(0.0, abs=1e-14)


def test_ks_statistic_hand_cases():
    assert stats.ks_statistic([1, 2, 3], [1, 2, 3]) == 0.0
    assert stats.ks_statistic([1, 2], [3, 4]) == 1.0
    # F_x jumps to 1/2 at 1 while F_y is 0 until 2: D = 1/2
    assert stats.ks_statistic([1, 3], [2, 3]) == pytest.approx(0.5)
    # identical maps: probability 1; disjoint samples of size 100: probability ~ 0
    assert stats.ks_probability(0.0, 100, 100) == pytest.approx(1.0)
    assert stats.ks_probability(1.0, 100, 100) < 1e-20


def test_ks_with_different_ray_densities():
    """With different N_rays the count-to-Delta-m maps differ: K-S must compare mu, not counts."""
    a = np.array([64, 64, 128, 128])            # mu = 1, 1, 2, 2 at N_rays = 64
    b = np.array([25, 50, 50, 50])              # mu = 1, 2, 2, 2 at N_rays = 25
    d = stats.ks_statistic(stats.delta_m(a, 64.0), stats.delta_m(b, 25.0))
    assert d == pytest.approx(0.25)
    assert stats.ks_statistic(a, b) == 1.0      # counts alone would say the samples are disjoint


def test_ks_of_counts_equals_ks_of_delta_m():
    """Delta m is strictly decreasing in the count, so the K-S statistic is the same on counts."""
    rng = np.random.default_rng(3)
    a = rng.poisson(30.0, 5000)
    b = rng.poisson(31.0, 5000)
    assert stats.ks_statistic(stats.delta_m(a, 30.0), stats.delta_m(b, 30.0)) == pytest.approx(
        stats.ks_statistic(a, b), abs=1e-15)


# Critical values of the Kolmogorov distribution, Q(lambda) = P(K > lambda), as tabulated by
# Smirnov (1948) and reprinted in standard statistical tables: the probability the K-S test of
# Sect. 3.1 reports at intermediate D, where neither 0 nor 1 pins it.
KOLMOGOROV_TABLE = [(0.20, 1.0727), (0.10, 1.2238), (0.05, 1.3581), (0.025, 1.4802), (0.01, 1.6276),
                    (0.005, 1.7308), (0.001, 1.9495)]


@pytest.mark.parametrize("na,nb", [(3000, 1500), (12, 6), (40, 10)])
def test_ks_probability_at_tabulated_kolmogorov_points(na, nb):
    """D is placed where the corrected argument (sqrt(n_e) + 0.12 + 0.11/sqrt(n_e)) D, with
    n_e = n_a n_b / (n_a + n_b), equals a tabulated critical value; the probability must equal that
    value's significance level. Unequal sample sizes make n_e differ from n_a, n_b, their sum or their
    geometric mean; n_e = 1000 makes the correction small but visible (a 0.4 % shift of the argument
    moves Q(1.3581) by 3 %), n_e = 4 and 8 make the 0.11/sqrt(n_e) term visible. The table's
    four decimals fix Q to about 5e-5."""
    ne = na * nb / (na + nb)
    for alpha, lam in KOLMOGOROV_TABLE:
        d = lam / (math.sqrt(ne) + 0.12 + 0.11 / math.sqrt(ne))
        assert stats.ks_probability(d, na, nb) == pytest.approx(alpha, abs=1e-4), (na, nb, alpha)
    # symmetric in the two samples
    assert stats.ks_probability(0.3, na, nb) == stats.ks_probability(0.3, nb, na)


def test_ks_probability_tracks_the_exact_two_sample_distribution():
    """The asymptotic form approximates the exact permutation distribution of the two-sample
    statistic (computed by scipy's exact method, a separate routine): within a quarter of its value
    for samples of 60 .. 300, where a wrong n_e would be off by one or more orders of magnitude."""
    from scipy import stats as ss
    rng = np.random.default_rng(5)
    for na, nb in [(40, 20), (60, 30), (200, 100)]:
        for shift in (0.0, 0.4, 0.8):
            x, y = rng.normal(0.0, 1.0, na), rng.normal(shift, 1.0, nb)
            r = ss.ks_2samp(x, y, method="exact")
            d = stats.ks_statistic(x, y)
            assert d == pytest.approx(r.statistic, abs=1e-15)
            p = stats.ks_probability(d, na, nb)
            if r.pvalue > 1e-3:
                assert abs(p - r.pvalue) <= 0.25 * r.pvalue, (na, nb, shift, p, r.pvalue)
