"""Pins of the oracle's far-field approximation (the tree code's idea on blocks of
rays, Sect. 2.1, Eq. hierarchical): each ray of a block sums its near lenses
exactly and takes the far lenses from P terms of the series about the block
centre. The pins are mathematics, not the oracle's own formulas:
  * one far lens: the P-term series is a truncated geometric series with a
    closed form;
  * every lens near: the direct sum of Eq. sigma, bit for bit;
  * many lenses: the error against the direct sum stays within the tail bound
    sum m t^P / (|d| (1 - t)), comes close to it, and shrinks as P grows.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import field

CFG0 = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=4.0, npix_side=128, nrays=100.0, margin=1.5)
CFG_SHEAR = dict(sigma=0.6, gamma=0.25, smooth_frac=0.3, side=4.0, npix_side=64, nrays=50.0, margin=1.5)


def field0():
    return synth.lens_field(100, field.radius_for_nstar(100, 0.4), 1)


def block_centre(g, i, j, bt, origin=(0, 0)):
    """Centre of the block of ray (i, j): blocks of 64 bt x 32 bt rays from the origin."""
    bw, bh = 64 * bt, 32 * bt
    ib = origin[0] + (i - origin[0]) // bw * bw
    jb = origin[1] + (j - origin[1]) // bh * bh
    return complex((ib + bw / 2 - g["nx"] / 2) * g["delta"], (jb + bh / 2 - g["ny"] / 2) * g["delta"])


@pytest.mark.parametrize("order", [1, 2, 5, 12])
def test_one_far_lens_is_a_truncated_geometric_series(order):
    g = oracle.geometry(CFG0)
    bt = 2
    rng = np.random.default_rng(order)
    ri = rng.integers(0, g["nx"], 64)
    rj = rng.integers(0, g["ny"], 64)
    for k in range(ri.size):
        zb = block_centre(g, ri[k], rj[k], bt)
        # one lens of mass 0.7 at 4 block radii from the block centre, in a random direction
        rho = g["delta"] * np.hypot(32 * bt, 16 * bt)
        zl = zb + 4 * rho * np.exp(1j * rng.uniform(0, 2 * np.pi))
        one = synth.LensField(np.array([zl.real]), np.array([zl.imag]), np.array([0.7]))
        a, _, _, b = oracle.far_rays(CFG0, one, dict(order=order, ratio=0.5, block_tiles=bt), ri[k:k + 1], rj[k:k + 1])
        z = complex((ri[k] + 0.5 - g["nx"] / 2) * g["delta"], (rj[k] + 0.5 - g["ny"] / 2) * g["delta"])
        w, d = z - zb, zl - zb
        # conj(alpha) = -m sum_{l<P} w^l / d^(l+1) = -m (1 - (w/d)^P) / (d - w)
        f = -0.7 * (1 - (w / d) ** order) / (d - w)
        assert a[0, 0] == pytest.approx(f.real, rel=1e-12, abs=1e-14)
        assert a[0, 1] == pytest.approx(-f.imag, rel=1e-12, abs=1e-14)
        t = abs(w) / abs(d)
        assert b[0] == pytest.approx(0.7 * t ** order / (abs(d) * (1 - t)), rel=1e-12)


@pytest.mark.parametrize("cfg", [CFG0, CFG_SHEAR], ids=["plain", "shear"])
def test_every_lens_near_gives_the_direct_sum_bit_for_bit(cfg):
    f = field0()
    far = dict(order=8, ratio=1e-9, block_tiles=4)           # rho / q covers the whole field
    exact, te = oracle.shoot_map(cfg, f)
    got, tg, bmax = oracle.far_map(cfg, f, far)
    assert np.array_equal(got, exact) and tg == te and bmax == 0.0
    g = oracle.geometry(cfg)
    rng = np.random.default_rng(3)
    ri, rj = rng.integers(0, g["nx"], 500), rng.integers(0, g["ny"], 500)
    a0, y0, p0 = oracle.shoot_rays(cfg, f, ri, rj)
    a1, y1, p1, b1 = oracle.far_rays(cfg, f, far, ri, rj)
    assert np.array_equal(a0, a1) and np.array_equal(p0, p1) and not b1.any()


def test_truncation_error_within_the_tail_bound_and_close_to_it():
    f = field0()
    g = oracle.geometry(CFG0)
    rng = np.random.default_rng(5)
    ri, rj = rng.integers(0, g["nx"], 3000), rng.integers(0, g["ny"], 3000)
    a0, _, _ = oracle.shoot_rays(CFG0, f, ri, rj)
    worst = []
    for order in (1, 2, 4, 8, 16):
        a, _, _, b = oracle.far_rays(CFG0, f, dict(order=order, ratio=0.6, block_tiles=8), ri, rj)
        err = np.hypot(*(a - a0).T)
        assert np.all(err <= b * (1 + 1e-9) + 1e-12), order
        if order <= 4:
            big = b > 1e-6
            assert (err[big] / b[big]).max() > 0.2, order          # the bound is not vacuous
        worst.append(err.max())
    assert all(worst[k + 1] < worst[k] for k in range(len(worst) - 1)) and worst[-1] < 1e-3 * worst[0]


def test_default_far_map_matches_the_direct_map():
    f = field0()
    exact, te = oracle.shoot_map(CFG0, f)
    got, tg, bmax = oracle.far_map(CFG0, f, dict(order=16, ratio=0.3, block_tiles=8))
    assert bmax < 1e-7
    assert tg["shot"] == te["shot"]
    assert int(np.abs(got.astype(np.int64) - exact).sum()) <= 2


def test_ragged_rectangle_counts_every_ray_once():
    f = field0()
    rect = (13, 1713, 7, 907)                                # not a multiple of the block size
    got, tg, _ = oracle.far_map(CFG0, f, dict(order=12, ratio=0.4, block_tiles=2), rect=rect)
    exact, te = oracle.shoot_map(CFG0, f, rect=rect)
    assert tg["shot"] == (rect[1] - rect[0]) * (rect[3] - rect[2]) == te["shot"]
    assert tg["inside"] + tg["out"] == tg["shot"] and int(got.sum()) == tg["inside"]
    assert int(np.abs(got.astype(np.int64) - exact).sum()) <= 4
    # rays of the rectangle, with its blocks counted from its origin
    g = oracle.geometry(CFG0)
    rng = np.random.default_rng(9)
    ri, rj = rng.integers(rect[0], rect[1], 400), rng.integers(rect[2], rect[3], 400)
    a0, _, _ = oracle.shoot_rays(CFG0, f, ri, rj)
    a1, _, _, b1 = oracle.far_rays(CFG0, f, dict(order=12, ratio=0.4, block_tiles=2), ri, rj, origin=rect[::2])
    assert np.all(np.hypot(*(a1 - a0).T) <= b1 * (1 + 1e-9) + 1e-12)
    assert g["nx"] > rect[1] and g["ny"] > rect[3]


@pytest.mark.parametrize("far", [dict(order=0, ratio=0.3, block_tiles=8), dict(order=8, ratio=0.0, block_tiles=8),
                                 dict(order=8, ratio=1.0, block_tiles=8), dict(order=8, ratio=0.3, block_tiles=0)])
def test_bad_far_parameters_rejected(far):
    with pytest.raises(ValueError):
        oracle.far_map(CFG0, field0(), far)
