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


# ---- grouped far lenses (the tree code's cells of distant lenses, Sect. 2.1) ----
# A field of 4000 lognormal lenses in a disc of 100 Einstein radii around a 10 x 10 R_E ray grid:
# blocks of 2 x 2 tiles (radius 1.1 R_E) see most lenses from far away, so many cells of the lens
# tree are grouped.
CFG_G = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=4.0, npix_side=64, nrays=16.0, margin=1.5)
FAR_G = dict(order=10, ratio=0.3, block_tiles=2)


def field_g():
    return synth.lens_field(4000, field.radius_for_nstar(4000, 0.4), 21, synth.MASS_LOGNORMAL)


def rays_g(n=600, seed=1):
    g = oracle.geometry(CFG_G)
    rng = np.random.default_rng(seed)
    return rng.integers(0, g["nx"], n), rng.integers(0, g["ny"], n)


def test_grouping_that_groups_no_cell_is_the_ungrouped_method_bit_for_bit():
    """theta -> 0: no cell is ever far enough, every leaf gives up its lenses one by one, and the
    near and one-by-one lists (each lens exactly once, in index order) are the ungrouped ones."""
    f = field_g()
    ri, rj = rays_g()
    au, _, pu, bu = oracle.far_rays(CFG_G, f, FAR_G, ri, rj)
    ag, _, pg, bg = oracle.far_rays(CFG_G, f, dict(FAR_G, group_order=8, group_theta=1e-9, group_leaf=3), ri, rj)
    assert np.array_equal(au, ag) and np.array_equal(pu, pg) and np.array_equal(bu, bg)
    mu, tu, bmu = oracle.far_map(CFG_G, f, FAR_G)
    mg, tg, bmg = oracle.far_map(CFG_G, f, dict(FAR_G, group_order=8, group_theta=1e-9, group_leaf=3))
    assert np.array_equal(mu, mg) and tu == tg and bmu == bmg


def test_grouped_series_converges_to_the_ungrouped_series():
    """With K = 64 multipole terms and theta = 0.5 the cells' expansions are exact to rounding
    (their remainder is below 0.5^64 of a cell's pull), so grouping changes the deflection by
    rounding only; with a monopole alone (K = 1) the same grouping visibly changes it."""
    f = field_g()
    ri, rj = rays_g()
    au, _, _, _ = oracle.far_rays(CFG_G, f, FAR_G, ri, rj)
    a64, _, _, _ = oracle.far_rays(CFG_G, f, dict(FAR_G, group_order=64, group_theta=0.5, group_leaf=16), ri, rj)
    a1, _, _, _ = oracle.far_rays(CFG_G, f, dict(FAR_G, group_order=1, group_theta=0.5, group_leaf=16), ri, rj)
    assert np.hypot(*(a64 - au).T).max() < 1e-12
    assert np.hypot(*(a1 - au).T).max() > 1e-3
    # small leaves next to a wide near disc (q = 0.1, rho / q = 11 rho): cells close to the block are
    # grouped only when all their lenses are far, so the near lenses stay exact
    near = dict(FAR_G, ratio=0.1)
    au, _, _, _ = oracle.far_rays(CFG_G, f, near, ri, rj)
    a64, _, _, _ = oracle.far_rays(CFG_G, f, dict(near, group_order=64, group_theta=0.5, group_leaf=1), ri, rj)
    assert np.hypot(*(a64 - au).T).max() < 1e-12


def test_grouped_error_within_its_bound_and_shrinking_with_the_order():
    """Against the direct sum of Eq. sigma, the grouped far field's error stays within its bound
    (series tail of the lenses taken one by one plus the double-series remainder of every grouped
    cell) for each multipole order, and both the error and the bound fall as K grows."""
    f = field_g()
    ri, rj = rays_g(800, 4)
    a0, _, _ = oracle.shoot_rays(CFG_G, f, ri, rj)
    errs, bounds = [], []
    for K in (2, 4, 8, 16, 64):
        for P in (1, 2, 3, 10):
            a, _, _, b = oracle.far_rays(CFG_G, f, dict(FAR_G, order=P, group_order=K, group_theta=0.5, group_leaf=16),
                                         ri, rj)
            err = np.hypot(*(a - a0).T)
            assert np.all(err <= b * (1 + 1e-9) + 1e-12), (K, P)
            if P == 10 and K < 64:
                errs.append(err.max())
                bounds.append(b.max())
    assert all(errs[k + 1] < errs[k] for k in range(3)) and all(bounds[k + 1] < bounds[k] for k in range(3))
    # every lens beyond rho / q in a grouped cell (q = 0.05, single-lens leaves): the bound is the
    # cells' remainders alone, the part in w (l >= P) included
    for P in (1, 2):
        a, _, _, b = oracle.far_rays(CFG_G, f, dict(FAR_G, ratio=0.05, order=P, group_order=64, group_theta=0.5,
                                                    group_leaf=1), ri, rj)
        err = np.hypot(*(a - a0).T)
        assert np.all(err <= b * (1 + 1e-9) + 1e-12), P
        assert (err / b).max() > 0.01, P                       # and it is not vacuous


def test_grouped_map_matches_the_direct_map():
    """The default-like grouping (P = 10, K = 24, theta = 0.3) leaves the map of the exact method
    unchanged up to a few rays, with a bound of about 1e-6 Einstein radii at this coarse block."""
    f = field_g()
    exact, te = oracle.shoot_map(CFG_G, f)
    got, tg, bmax = oracle.far_map(CFG_G, f, dict(FAR_G, group_order=24, group_theta=0.3, group_leaf=32))
    assert tg == te and bmax < 1e-5
    assert int(np.abs(got.astype(np.int64) - exact).sum()) <= 8


@pytest.mark.parametrize("extra", [dict(group_order=65, group_theta=0.5, group_leaf=8),
                                   dict(group_order=8, group_theta=0.0, group_leaf=8),
                                   dict(group_order=8, group_theta=1.0, group_leaf=8),
                                   dict(group_order=8, group_theta=0.5, group_leaf=0)])
def test_bad_grouping_parameters_rejected(extra):
    with pytest.raises(ValueError):
        oracle.far_map(CFG0, field0(), dict(order=8, ratio=0.3, block_tiles=8, **extra))
