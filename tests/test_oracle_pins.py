"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Every check here is independent of the oracle's own code: printed numbers
from the paper (golden files), exact rational arithmetic, a textbook closed
form, and invariants. Each is chosen so that a plausible mistake in the
oracle (a dropped smooth or shear term, a wrong sign, a transposed map, a
wrong lattice offset, a mass ignored) fails at least one of them.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
import synth
from oracle import field

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ---------------------------------------------------------------- Eq. nstar ----

def test_nstar_rule_reproduces_printed_sweeps():
    """Sect. 3.1 prints N* for the sigma and gamma sweeps; the disc reading + Eq. nstar
    must give them exactly, except sigma = 0.9 which is printed 0.02 % lower."""
    exact = 0
    for sweep, s, g, printed in _rows("nstar_sweeps.txt"):
        n, _ = field.nstar_rule(float(s), float(g), 0.0, 20.0)
        if int(printed) == n:
            exact += 1
        else:
            assert (sweep, s) == ("sigma", "0.9"), (sweep, s, g, printed, n)
            assert abs(n - int(printed)) / int(printed) < 5e-4
    assert exact == 19


def test_nstar_radius_roundtrip_and_lognormal_mean():
    r = field.radius_for_nstar(25000, 0.4)
    assert abs(r - 250.0) < 1e-12
    assert field.nstar_for_radius(0.4, r) == 25000
    assert abs(field.mean_mass(1, 0.0, 0.5) - math.exp(0.125)) < 1e-15
    # <M> = E[exp(N(0, 0.25))] by a seeded sample of the generator's lognormal masses
    m = synth.masses(400000, 7, synth.MASS_LOGNORMAL, 0.0, 0.5)
    assert abs(m.mean() / field.mean_mass(1, 0.0, 0.5) - 1.0) < 5e-3


# ------------------------------------------------------------- Eq. mutheory ----

def test_mu_theory_printed_values():
    for _, s, g, printed, digits in _rows("mu_av.txt"):
        v = field.mu_theory(float(s), float(g))
        assert round(v, int(digits)) == pytest.approx(float(printed), abs=0.5 * 10 ** -int(digits))


# -------------------------------------------------- smooth-only closed form ----

def _lattice_counts_1d(coef: Fr, n_rays_1d: int, delta: Fr, pix: Fr, nside: int):
    """Exact number of lattice columns whose source coordinate coef * x_i falls in each pixel,
    and the smallest distance (in pixels) of any such coordinate from a pixel edge."""
    counts = np.zeros(nside, dtype=np.int64)
    mind = Fr(10 ** 9)
    half = Fr(nside, 2)
    for i in range(n_rays_1d):
        x = (Fr(2 * i + 1, 2) - Fr(n_rays_1d, 2)) * delta
        u = coef * x / pix + half
        k = math.floor(u)
        mind = min(mind, u - k, k + 1 - u)
        if 0 <= k < nside:
            counts[k] += 1
    return counts, mind


def test_smooth_only_map_is_exact_closed_form():
    """N* = 0 with all matter smooth (s = 1): the lens equation is diagonal, y = diag(a, b) x,
    so pixel (I, J) receives (#columns mapped into I) x (#rows mapped into J) rays, exactly."""
    sigma, gamma = Fr("0.53"), Fr("0.1")
    side, nside, nrays, margin = Fr(2), 16, 121, Fr("1.5")
    p = dict(sigma=0.53, gamma=0.1, smooth_frac=1.0, side=2.0, npix_side=nside, nrays=121.0, margin=1.5)
    a, b = 1 - sigma - gamma, 1 - sigma + gamma
    pix = side / nside
    delta = pix / 11                                  # sqrt(121) = 11
    w, h = margin * side / abs(a), margin * side / abs(b)
    nx, ny = math.ceil(w / delta), math.ceil(h / delta)
    assert min(w / delta - math.floor(w / delta), h / delta - math.floor(h / delta)) > Fr(1, 100)
    g = oracle.geometry(p)
    assert (g["nx"], g["ny"]) == (nx, ny)

    cols, dcol = _lattice_counts_1d(a, nx, delta, pix, nside)
    rows, drow = _lattice_counts_1d(b, ny, delta, pix, nside)
    assert min(dcol, drow) > Fr(1, 10 ** 6)           # no ray within 1e-6 px of an edge
    expect = np.outer(rows, cols)

    empty = synth.lens_field(0, 1.0, 0)
    got, tot = oracle.shoot_map(p, empty)
    np.testing.assert_array_equal(got.astype(np.int64), expect)
    assert tot["shot"] == nx * ny
    assert tot["inside"] == int(expect.sum())
    assert tot["shot"] == tot["inside"] + tot["out"]
    # mean magnification over the map -> |mu_av| (Eq. mutheory), up to one lattice line per side
    mu_map = got.mean() / nrays
    mu_av = abs(field.mu_theory(0.53, 0.1))
    assert abs(mu_map / mu_av - 1.0) < 0.01


def test_smooth_only_transposes_with_shear_sign():
    """Flipping the sign of the shear swaps the roles of the axes: the map transposes."""
    base = dict(sigma=0.53, smooth_frac=1.0, side=2.0, npix_side=16, nrays=121.0, margin=1.5)
    empty = synth.lens_field(0, 1.0, 0)
    m1, _ = oracle.shoot_map(dict(base, gamma=0.1), empty)
    m2, _ = oracle.shoot_map(dict(base, gamma=-0.1), empty)
    np.testing.assert_array_equal(m1, m2.T)
    assert not np.array_equal(m1, m1.T)


# --------------------------------------------------------------- point lens ----

def _point_lens_mu(u):
    """Total magnification of a point lens for a source at distance u (Einstein radii)."""
    return (u * u + 2.0) / (u * np.sqrt(u * u + 4.0))


def test_single_point_lens_matches_analytic_magnification():
    """N* = 1 unit mass at the origin, no smooth matter or shear: N_IJ / N_rays must equal the
    point-lens magnification averaged over the pixel (textbook closed form)."""
    nside, side, nrays = 16, 4.0, 10000.0
    p = dict(sigma=0.0, gamma=0.0, smooth_frac=0.0, side=side, npix_side=nside, nrays=nrays, margin=1.5)
    lens = synth.LensField(np.array([0.0]), np.array([0.0]), np.array([1.0]))
    got, tot = oracle.shoot_map(p, lens)
    pix = side / nside
    q = (np.arange(64) + 0.5) / 64.0
    checked = 0
    for J in range(nside):
        for I in range(nside):
            y1 = -side / 2 + (I + q[None, :]) * pix
            y2 = -side / 2 + (J + q[:, None]) * pix
            u = np.hypot(y1, y2)
            if u.min() < 2 * pix or u.max() > 2.2:      # near the caustic point / image outside the grid
                continue
            expect = _point_lens_mu(u).mean()
            assert abs(got[J, I] / nrays / expect - 1.0) < 0.03, (I, J, got[J, I] / nrays, expect)
            checked += 1
    assert checked >= 100
    assert tot["shot"] == tot["inside"] + tot["out"]


def test_single_lens_mass_scales_einstein_radius():
    """A lens of mass m is a unit lens with lengths scaled by sqrt(m): the map of mass 4 on side
    2L equals the map of mass 1 on side L, pixel for pixel, up to rays within rounding of an edge."""
    base = dict(sigma=0.0, gamma=0.0, smooth_frac=0.0, npix_side=12, nrays=400.0, margin=1.5)
    m1, _ = oracle.shoot_map(dict(base, side=3.0), synth.LensField(np.array([0.0]), np.array([0.0]), np.array([1.0])))
    m4, _ = oracle.shoot_map(dict(base, side=6.0), synth.LensField(np.array([0.0]), np.array([0.0]), np.array([4.0])))
    diff = np.abs(m1.astype(np.int64) - m4.astype(np.int64)).sum()
    assert diff <= 2e-6 * m1.sum() + 4


# ----------------------------------------------------- brute force, exact -----

def _exact_pixel(x1, x2, lenses, sigma_c, gamma, side, pix, nside):
    a1 = a2 = Fr(0)
    for lx, ly, lm in lenses:
        d1, d2 = x1 - lx, x2 - ly
        r2 = d1 * d1 + d2 * d2
        a1 += lm * d1 / r2
        a2 += lm * d2 / r2
    y1 = (1 - gamma) * x1 - sigma_c * x1 - a1
    y2 = (1 + gamma) * x2 - sigma_c * x2 - a2
    u1 = (y1 + side / 2) / pix
    u2 = (y2 + side / 2) / pix
    k1, k2 = math.floor(u1), math.floor(u2)
    dist = min(u1 - k1, k1 + 1 - u1, u2 - k2, k2 + 1 - u2)
    if 0 <= k1 < nside and 0 <= k2 < nside:
        return k2 * nside + k1, dist, (a1, a2)
    return -1, dist, (a1, a2)


def test_brute_force_exact_rational_tiny_map():
    """3 lenses of unequal mass, smooth matter and shear, a 4 x 4 map: every ray recomputed in
    exact rational arithmetic must land in the oracle's pixel, and the maps must be identical."""
    sigma, gamma, s = Fr("0.4"), Fr("0.25"), Fr("0.5")
    side, nside, nrays = Fr(2), 4, 100
    p = dict(sigma=0.4, gamma=0.25, smooth_frac=0.5, side=2.0, npix_side=nside, nrays=100.0, margin=1.5)
    f = synth.lens_field(3, 2.5, 11)
    f.m = np.array([0.5, 1.0, 2.0])
    lenses = [(Fr(float(x)), Fr(float(y)), Fr(float(m))) for x, y, m in zip(f.x, f.y, f.m)]
    pix = side / nside
    delta = pix / 10
    a, b = 1 - sigma - gamma, 1 - sigma + gamma
    nx = math.ceil(Fr("1.5") * side / abs(a) / delta)
    ny = math.ceil(Fr("1.5") * side / abs(b) / delta)
    g = oracle.geometry(p)
    assert (g["nx"], g["ny"]) == (nx, ny)

    expect = np.zeros(nside * nside, dtype=np.int64)
    ii, jj, pe, al = [], [], [], []
    mind = Fr(1)
    for j in range(ny):
        x2 = (Fr(2 * j + 1, 2) - Fr(ny, 2)) * delta
        for i in range(nx):
            x1 = (Fr(2 * i + 1, 2) - Fr(nx, 2)) * delta
            k, dist, alpha = _exact_pixel(x1, x2, lenses, s * sigma, gamma, side, pix, nside)
            mind = min(mind, dist)
            if k >= 0:
                expect[k] += 1
            if (i * 7 + j * 13) % 97 == 0:
                ii.append(i); jj.append(j); pe.append(k); al.append((float(alpha[0]), float(alpha[1])))
    assert mind > Fr(1, 10 ** 9)
    got, tot = oracle.shoot_map(p, f)
    np.testing.assert_array_equal(got.reshape(-1).astype(np.int64), expect)
    assert tot["shot"] == nx * ny and tot["inside"] == int(expect.sum())
    alpha, _, pix_o = oracle.shoot_rays(p, f, ii, jj)
    np.testing.assert_array_equal(pix_o, np.array(pe))
    np.testing.assert_allclose(alpha, np.array(al), rtol=1e-12, atol=1e-13)


# --------------------------------------------------------------- invariants ----

def _small_field_params():
    p = dict(sigma=0.45, gamma=0.2, smooth_frac=0.3, side=3.0, npix_side=32, nrays=64.0, margin=1.5)
    n, r = field.nstar_rule(p["sigma"], p["gamma"], p["smooth_frac"], p["side"])
    return p, synth.lens_field(n, r, 5)


def test_conservation_and_subrectangles_add_up():
    p, f = _small_field_params()
    full, tot = oracle.shoot_map(p, f)
    g = oracle.geometry(p)
    assert tot["shot"] == g["nx"] * g["ny"] == tot["inside"] + tot["out"]
    assert int(full.sum(dtype=np.int64)) == tot["inside"]
    h = g["ny"] // 3
    lo, tlo = oracle.shoot_map(p, f, rect=(0, g["nx"], 0, h))
    hi, thi = oracle.shoot_map(p, f, rect=(0, g["nx"], h, g["ny"]))
    np.testing.assert_array_equal(lo.astype(np.int64) + hi, full)
    assert tlo["shot"] + thi["shot"] == tot["shot"]


def test_mirror_symmetry_of_field_mirrors_map():
    """Reflecting every lens x -> -x reflects the map left-right (the ray grid is symmetric)."""
    p, f = _small_field_params()
    m1, t1 = oracle.shoot_map(p, f)
    m2, t2 = oracle.shoot_map(p, synth.LensField(-f.x, f.y.copy(), f.m.copy()))
    diff = np.abs(m1.astype(np.int64) - m2[:, ::-1]).sum()
    assert diff <= 4 and t1["shot"] == t2["shot"]


def test_ray_on_a_lens_is_out():
    p = dict(sigma=0.0, gamma=0.0, smooth_frac=0.0, side=2.0, npix_side=4, nrays=16.0, margin=1.5)
    g = oracle.geometry(p)
    x1 = (3 + 0.5 - 0.5 * g["nx"]) * g["delta"]
    x2 = (5 + 0.5 - 0.5 * g["ny"]) * g["delta"]
    lens = synth.LensField(np.array([x1]), np.array([x2]), np.array([1.0]))
    _, _, pix = oracle.shoot_rays(p, lens, [3, 4], [5, 5])
    assert pix[0] == -1 and pix[1] >= -1


def test_threads_do_not_change_the_map():
    p, f = _small_field_params()
    a, _ = oracle.shoot_map(p, f, threads=1)
    b, _ = oracle.shoot_map(p, f, threads=4)
    np.testing.assert_array_equal(a, b)


def test_ill_posed_parameters_rejected():
    with pytest.raises(ValueError):
        oracle.geometry(dict(sigma=0.5, gamma=0.5, smooth_frac=0.0, side=2.0, npix_side=8, nrays=10.0))
