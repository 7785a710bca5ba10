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
