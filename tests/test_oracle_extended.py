"""Pins of the oracle's extended-source convolution and light curves (Sect. 1)."""
import math

import numpy as np
import pytest

from oracle import extended as ext


def test_uniform_map_stays_uniform():
    c = np.full((40, 40), 300)
    for prof, size in ((0, 0.05), (1, 0.12)):
        out = ext.convolve(c, 100.0, prof, size, 0.02)
        v = out[~np.isnan(out)]
        assert v.size > 0 and np.allclose(v, 3.0, rtol=0, atol=1e-12)


def test_disc_support_is_the_gauss_circle_count():
    # lattice points with i^2 + j^2 <= r^2: 13 (r = 2), 29 (r = 3), 81 (r = 5) -- Gauss's circle problem
    for r, count in ((2, 13), (3, 29), (5, 81)):
        w = ext.profile_weights(1, r * 0.1, 0.1)
        assert int(np.count_nonzero(w)) == count
        assert w.sum() == pytest.approx(1.0)


def test_point_map_reproduces_the_profile():
    n, pix, s = 81, 0.01, 0.03
    c = np.zeros((n, n))
    c[40, 40] = 1.0
    out = ext.convolve(c, 1.0, 0, s, pix)
    h = math.ceil(4 * s / pix)
    k = np.arange(-h, h + 1) * pix
    g = np.exp(-k * k / (2 * s * s))
    ref = np.outer(g, g) / np.outer(g, g).sum()
    np.testing.assert_allclose(out[40 - h:41 + h, 40 - h:41 + h], ref[::-1, ::-1], rtol=1e-12, atol=1e-15)
    assert np.isnan(out[0, 0]) and np.isnan(out[40, h - 1]) and not np.isnan(out[40, h])


def test_lightcurve_is_exact_on_a_plane():
    n, side = 32, 3.2
    jj, ii = np.mgrid[0:n, 0:n]
    plane = 2.0 + 0.5 * ii - 0.25 * jj                  # bilinear interpolation is exact on planes
    lc = ext.lightcurve(plane, side, (-1.0, -0.7), (1.1, 0.9), 57)
    t = np.linspace(0, 1, 57)
    y1 = -1.0 + t * 2.1
    y2 = -0.7 + t * 1.6
    u = (y1 + side / 2) / (side / n) - 0.5
    v = (y2 + side / 2) / (side / n) - 0.5
    np.testing.assert_allclose(lc, 2.0 + 0.5 * u - 0.25 * v, rtol=1e-12)
    assert np.isnan(ext.lightcurve(plane, side, (-1.6, 0.0), (-1.6, 0.0), 1)[0])


def test_convolve_at_pixels_equals_the_whole_convolution():
    """convolve_at (the oracle's convolution at listed pixels, for maps too large to convolve whole)
    against convolve() on a seeded map: equal within FP64 rounding, NaN alike near the edges."""
    rng = np.random.default_rng(3)
    c = rng.poisson(30.0, (48, 48))
    for prof, size in ((0, 0.05), (1, 0.12)):
        full = ext.convolve(c, 30.0, prof, size, 0.02)
        jj, ii = np.mgrid[0:48, 0:48]
        got = ext.convolve_at(c, 30.0, prof, size, 0.02, ii.ravel(), jj.ravel()).reshape(48, 48)
        np.testing.assert_array_equal(np.isnan(got), np.isnan(full))
        ok = ~np.isnan(full)
        np.testing.assert_allclose(got[ok], full[ok], rtol=1e-13, atol=0)


def test_convolve_at_keeps_the_pins():
    """The pins of convolve() hold for convolve_at: a uniform map stays uniform and a point map
    reproduces the normalised profile around the point."""
    c = np.full((40, 40), 300)
    assert np.allclose(ext.convolve_at(c, 100.0, 1, 0.12, 0.02, [20, 10], [20, 30]), 3.0, rtol=0, atol=1e-12)
    n, pix, s = 81, 0.01, 0.03
    p = np.zeros((n, n))
    p[40, 40] = 1.0
    h = math.ceil(4 * s / pix)
    w = ext.profile_weights(0, s, pix)
    got = ext.convolve_at(p, 1.0, 0, s, pix, [40 + 3, 40 - 5], [40 - 2, 40 + 7])
    np.testing.assert_allclose(got, [w[h + 2, h - 3], w[h - 7, h + 5]], rtol=1e-12, atol=0)


def test_lightcurve_of_counts_equals_sampling_the_convolved_map():
    rng = np.random.default_rng(8)
    c = rng.poisson(50.0, (40, 40))
    side = 4.0
    for prof, size in ((0, 0.12), (1, 0.3)):
        full = ext.convolve(c, 50.0, prof, size, side / 40)
        start, end = (-1.9, -1.2), (1.7, 1.95)          # runs off the valid region at both ends
        ref = ext.lightcurve(full, side, start, end, 83)
        got = ext.lightcurve_of_counts(c, 50.0, prof, size, side, start, end, 83)
        np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
        ok = ~np.isnan(ref)
        assert 20 < ok.sum() < 83
        np.testing.assert_allclose(got[ok], ref[ok], rtol=1e-13, atol=0)
