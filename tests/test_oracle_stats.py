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
