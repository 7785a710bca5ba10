"""Pins of the oracle's random rays (the paper's GPU code shoots rays from pseudo-random positions,
Sect. 2.3 step 2, so that a pixel receives N_rays rays only on average, Sect. 3.1).

Reading taken: the same nx * ny rays as the lattice, ray (i, j) uniform in the 64 x 32-cell tile of
the lattice that holds cell (i, j), its two fractions the top 18 bits of outputs 2q + 1 and 2q + 2
(q = j nx + i) of SplitMix64(ray_seed).

What pins it, without retyping the oracle's arithmetic:
- the positions against SplitMix64 outputs from the input module's own implementation (synth);
- uniformity and independence of the positions within their tiles (K-S and correlations);
- Poisson pixel counts of a lens-free map (mean N_rays exactly, variance equal to the mean), which the
  regular lattice does not have (variance 0);
- a random-ray map differs from the lattice map of the same lensed field by the Poisson noise of
  independent rays, and, where that noise is small, the two agree by the paper's criterion (RMS of
  Delta m below 0.2 mag, K-S probability above 99.7 %; Sect. 3.1). At N_rays = 100 on 128^2 pixels
  the K-S test already tells them apart (p ~ 1e-20): the noise of random rays is insignificant only
  at the paper's large ray counts.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import field
from oracle import stats as ostats

SEED = 12345
# sigma = gamma = 0 and no lenses: the lens equation is the identity, y = x
IDENTITY = dict(sigma=0.0, gamma=0.0, smooth_frac=0.0, side=2.0, npix_side=16, nrays=16.0,
                ray_mode=oracle.RAYS_RANDOM, ray_seed=SEED)
NO_LENSES = synth.lens_field(0, 1.0, 1)


def positions(p):
    """Ray positions of the whole grid from the oracle (the identity map returns them as y)."""
    g = oracle.geometry(p)
    jj, ii = np.meshgrid(np.arange(g["ny"]), np.arange(g["nx"]), indexing="ij")
    ri, rj = ii.ravel(), jj.ravel()
    _, y, _ = oracle.shoot_rays(p, NO_LENSES, ri, rj)
    return g, ri, rj, y


def test_random_positions_follow_splitmix64_and_the_tiles():
    g, ri, rj, y = positions(IDENTITY)
    assert (g["nx"], g["ny"]) == (96, 96)                  # one partial tile column (32 cells wide)
    q = (rj.astype(np.uint64) * np.uint64(g["nx"]) + ri.astype(np.uint64))
    z1 = synth.splitmix64(SEED, 2 * q + np.uint64(1))
    z2 = synth.splitmix64(SEED, 2 * q + np.uint64(2))
    u1 = (z1 >> np.uint64(46)).astype(np.float64) / 262144.0
    u2 = (z2 >> np.uint64(46)).astype(np.float64) / 262144.0
    ti, tj = ri // 64, rj // 32
    wi = np.minimum(64, g["nx"] - 64 * ti).astype(np.float64)
    wj = np.minimum(32, g["ny"] - 32 * tj).astype(np.float64)
    x1 = ((64 * ti).astype(np.float64) + u1 * wi - 0.5 * g["nx"]) * g["delta"]
    x2 = ((32 * tj).astype(np.float64) + u2 * wj - 0.5 * g["ny"]) * g["delta"]
    np.testing.assert_array_equal(y[:, 0], x1)
    np.testing.assert_array_equal(y[:, 1], x2)
    _, _, _, yl = positions(dict(IDENTITY, ray_mode=oracle.RAYS_LATTICE))
    assert np.abs(yl - y).max() > 10 * g["delta"]          # the mode changes the positions
    other = positions(dict(IDENTITY, ray_seed=SEED + 1))[3]
    assert (other != y).mean() > 0.99                      # and so does the seed


def test_random_rays_are_uniform_and_independent_in_their_tiles():
    from scipy import stats
    p = dict(IDENTITY, nrays=400.0)
    g, ri, rj, y = positions(p)
    cx = y[:, 0] / g["delta"] + 0.5 * g["nx"]                # position in cells from the grid corner
    cy = y[:, 1] / g["delta"] + 0.5 * g["ny"]
    ti, tj = ri // 64, rj // 32
    wi = np.minimum(64, g["nx"] - 64 * ti)
    wj = np.minimum(32, g["ny"] - 32 * tj)
    f1 = (cx - 64 * ti) / wi
    f2 = (cy - 32 * tj) / wj
    assert f1.min() >= 0.0 and f1.max() < 1.0 and f2.min() >= 0.0 and f2.max() < 1.0
    assert (wi < 64).any()                                 # partial tiles are spread over their width
    n = f1.size
    assert stats.kstest(f1, "uniform").pvalue > 1e-4
    assert stats.kstest(f2, "uniform").pvalue > 1e-4
    assert stats.kstest(f1[wi < 64], "uniform").pvalue > 1e-4
    lim = 5.0 / np.sqrt(n)
    assert abs(np.corrcoef(f1, f2)[0, 1]) < lim
    assert abs(np.corrcoef(f1[1:], f1[:-1])[0, 1]) < lim    # neighbouring rays
    assert abs(np.corrcoef(f2[1:], f2[:-1])[0, 1]) < lim


def test_lens_free_random_map_has_poisson_counts():
    """Every map pixel lies inside the shot rectangle, so its expected count is N_rays exactly; random
    rays make it (close to) Poisson, the lattice makes it exact."""
    p = dict(IDENTITY, npix_side=64, nrays=25.0, side=4.0)
    counts, tot = oracle.shoot_map(p, NO_LENSES)
    g = oracle.geometry(p)
    assert tot["shot"] == g["nx"] * g["ny"] and tot["inside"] + tot["out"] == tot["shot"]
    assert int(counts.sum()) == tot["inside"]
    c = counts.astype(np.float64).ravel()
    npix = c.size
    assert abs(c.mean() - 25.0) < 4.0 * np.sqrt(25.0 / npix)
    assert abs(c.var() / c.mean() - 1.0) < 4.0 * np.sqrt(2.0 / npix)
    lat, _ = oracle.shoot_map(dict(p, ray_mode=oracle.RAYS_LATTICE), NO_LENSES)
    assert (lat == 25).all()


CFG0 = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=4.0)     # BASELINE config 0's field


@pytest.fixture(scope="module")
def field0():
    return synth.lens_field(100, field.radius_for_nstar(100, 0.4), 1)


def test_random_map_differs_from_the_lattice_map_by_poisson_noise(field0):
    """Per pixel, the random map's count differs from the lattice map's by the noise of independent
    rays: Delta m moves by about (2.5 / ln 10) / sqrt(N_ij), so the RMS difference is close to
    1.0857 sqrt(mean 1 / N_ij) (a little below it, since the count in a tile is fixed)."""
    p = dict(CFG0, npix_side=64, nrays=400.0)
    lat, tl = oracle.shoot_map(p, field0)
    rnd, tr = oracle.shoot_map(dict(p, ray_mode=oracle.RAYS_RANDOM, ray_seed=SEED), field0)
    assert tl["shot"] == tr["shot"]
    st = ostats.compare(lat, 400.0, rnd, 400.0)
    pred = 2.5 / np.log(10.0) * np.sqrt(np.mean(1.0 / lat[lat > 0]))
    assert 0.85 < st["rms_dm"] / pred < 1.05
    assert (lat != rnd).mean() > 0.9


def test_random_and_lattice_maps_agree_excellently(field0):
    """The paper's criterion (Sect. 3.1: RMS of Delta m below 0.2 mag and a K-S probability above
    99.7 %) between a regular-grid map and a random-ray map of the same lensed field, at a ray count
    where the Poisson noise is small (N_rays = 4000 on 32^2 pixels)."""
    p = dict(CFG0, npix_side=32, nrays=4000.0)
    lat, _ = oracle.shoot_map(p, field0)
    rnd, _ = oracle.shoot_map(dict(p, ray_mode=oracle.RAYS_RANDOM, ray_seed=SEED), field0)
    st = ostats.compare(lat, 4000.0, rnd, 4000.0)
    assert st["rms_dm"] < 0.2
    assert st["ks_p"] > 0.997
    assert abs(st["mean_mu_a"] - st["mean_mu_b"]) < 0.01 * st["mean_mu_a"]


def test_far_field_rejects_random_rays():
    far = dict(order=4, ratio=0.3, block_tiles=1)
    with pytest.raises(ValueError):
        oracle.far_map(IDENTITY, NO_LENSES, far)
