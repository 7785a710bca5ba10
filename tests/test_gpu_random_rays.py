"""Random rays on the device (mm_params.ray_mode = MM_RAYS_RANDOM), as the paper's GPU code shoots
them (Sect. 2.3, step 2), against the oracle's random rays: the same positions, hence the same
tolerances as the lattice (see test_gpu_parity.py): per-ray |d alpha| <= 1e-5 R_E and <= 1e-4 of the
rays in another pixel for the FP32 path; FP64 within rounding; exact ray totals. Also: the noise
of random rays against the lattice map (the paper's excellent agreement where it is small),
batches that mix ray modes, maps in parts, and the calls that take the lattice only."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_1005_5198_gb300 as mm
import synth
from oracle import field

pytestmark = pytest.mark.gpu

ALPHA_TOL = 1e-5
MISBIN_TOL = 1e-4
SEED = 777
CFG0 = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=4.0, npix_side=128, nrays=100.0)
CFG2 = dict(sigma=0.8, gamma=0.3, smooth_frac=0.5, side=40.0, npix_side=2048, nrays=500.0)
RND = dict(ray_mode=mm.MM_RAYS_RANDOM, ray_seed=SEED)
ORND = dict(ray_mode=oracle.RAYS_RANDOM, ray_seed=SEED, margin=1.5)


@pytest.fixture(scope="module")
def ctx():
    mm.build()
    c = mm.mm_init(0)
    yield c
    mm.mm_destroy(c)


@pytest.fixture(scope="module")
def f0():
    return synth.lens_field(100, field.radius_for_nstar(100, 0.4), 1)


def P(cfg, **kw):
    d = dict(cfg)
    d.update(kw)
    return mm.params(**d)


def shoot(ctx, lh, p):
    m = mm.mm_shoot(ctx, lh, p)
    counts, st = mm.mm_map_fetch(ctx, m)
    mm.mm_release_map(ctx, m)
    return counts, st


def map_l1(a, b):
    return int(np.abs(a.astype(np.int64) - b.astype(np.int64)).sum())


def check_totals(counts, st, shot):
    assert st["rays_shot"] == shot
    assert st["rays_in"] + st["rays_out"] == shot
    assert int(counts.sum(dtype=np.int64)) == st["rays_in"]


def test_random_fp32_map_and_every_ray_match_oracle(ctx, f0):
    lh = mm.mm_create_lenses_from(ctx, f0.x, f0.y, f0.m)
    got, st = shoot(ctx, lh, P(CFG0, **RND))
    ref, tot = oracle.shoot_map(dict(CFG0, **ORND), f0)
    check_totals(got, st, tot["shot"])
    assert map_l1(got, ref) <= 2 * MISBIN_TOL * tot["shot"]
    lat, _ = shoot(ctx, lh, P(CFG0))
    assert map_l1(got, lat) > 0.02 * tot["inside"]         # Poisson noise: about 0.8 sqrt(N) per pixel
    g = oracle.geometry(dict(CFG0, **ORND))
    jj, ii = np.meshgrid(np.arange(g["ny"]), np.arange(g["nx"]), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    a_g, p_g = mm.mm_debug_deflect(ctx, lh, P(CFG0, **RND), ii, jj)
    a_o, _, p_o = oracle.shoot_rays(dict(CFG0, **ORND), f0, ii, jj)
    err = np.hypot(a_g[:, 0] - a_o[:, 0], a_g[:, 1] - a_o[:, 1])
    print(f"random rays, every ray of config 0: max |d alpha| {err.max():.3e}, misbinned {np.mean(p_g != p_o):.3e}")
    assert err.max() <= ALPHA_TOL
    assert np.mean(p_g != p_o) <= MISBIN_TOL


def test_random_fp64_matches_oracle(ctx, f0):
    lh = mm.mm_create_lenses_from(ctx, f0.x, f0.y, f0.m)
    got, st = shoot(ctx, lh, P(CFG0, precision=mm.MM_FP64, **RND))
    ref, tot = oracle.shoot_map(dict(CFG0, **ORND), f0)
    check_totals(got, st, tot["shot"])
    assert map_l1(got, ref) <= 2 * max(1, 1e-8 * tot["shot"])
    rng = np.random.default_rng(3)
    g = oracle.geometry(dict(CFG0, **ORND))
    ii, jj = rng.integers(0, g["nx"], 20000), rng.integers(0, g["ny"], 20000)
    a_g, p_g = mm.mm_debug_deflect(ctx, lh, P(CFG0, precision=mm.MM_FP64, **RND), ii, jj)
    a_o, _, p_o = oracle.shoot_rays(dict(CFG0, **ORND), f0, ii, jj)
    assert np.all(np.abs(a_g - a_o) <= 1e-9 * (1 + np.abs(a_o)))
    assert np.sum(p_g != p_o) <= 1


def test_random_split_tiles_match_oracle(ctx):
    """A tile-aligned window of the N* = 25 000 map: each tile's lens sum is split over CTAs."""
    f = synth.lens_field(25000, field.radius_for_nstar(25000, 0.4), 3)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    g = oracle.geometry(dict(CFG2, **ORND))
    i0, j0 = (g["nx"] // 3) // 64 * 64, (g["ny"] // 2) // 32 * 32
    rect = (i0, i0 + 577, j0, j0 + 389)
    m = mm.mm_shoot(ctx, lh, P(CFG2, ray_rect=rect, **RND))
    got, st = mm.mm_map_fetch(ctx, m)
    mm.mm_release_map(ctx, m)
    assert st["lens_splits"] > 1
    ref, tot = oracle.shoot_map(dict(CFG2, **ORND), f, rect=rect)
    check_totals(got, st, tot["shot"])
    assert map_l1(got, ref) <= 2 * max(2, MISBIN_TOL * tot["shot"])
    rng = np.random.default_rng(9)
    ii, jj = rng.integers(rect[0], rect[1], 4000), rng.integers(rect[2], rect[3], 4000)
    a_g, p_g = mm.mm_debug_deflect(ctx, lh, P(CFG2, ray_rect=rect, **RND), ii, jj)
    a_o, _, p_o = oracle.shoot_rays(dict(CFG2, **ORND), f, ii, jj)
    err = np.hypot(a_g[:, 0] - a_o[:, 0], a_g[:, 1] - a_o[:, 1])
    assert err.max() <= ALPHA_TOL and np.mean(p_g != p_o) <= MISBIN_TOL


def restore(ctx, lh, cfg, counts, tot, nstar):
    """A map on the device holding the oracle's counts and totals (mm_map_restore)."""
    g = mm.mm_geometry_of(P(cfg))
    st = dict(rays_shot=tot["shot"], rays_in=tot["inside"], rays_out=tot["out"], interactions=0, nx=g["nx"],
              ny=g["ny"], nstar=nstar, seconds=0.0, mu_mean=0.0, lens_splits=1, far_bound=0.0, far_block=0)
    return mm.mm_map_restore(ctx, lh, P(cfg), counts, st)


def test_random_and_lattice_maps_agree_excellently_on_the_device(ctx, f0):
    """The paper's comparison of a random-ray map with a regular-grid map of the same field (Sect. 3.1),
    made on the device by mm_map_compare, where the noise of random rays is small (32^2, N_rays = 4000):
    RMS of Delta m below 0.2 and a K-S probability above 99.7 %. The device's statistics of the
    oracle's two maps (put on the device by mm_map_restore) equal the oracle's statistics of them."""
    lh = mm.mm_create_lenses_from(ctx, f0.x, f0.y, f0.m)
    cfg = dict(CFG0, npix_side=32, nrays=4000.0)
    a = mm.mm_shoot(ctx, lh, P(cfg))
    b = mm.mm_shoot(ctx, lh, P(cfg, **RND))
    st = mm.mm_map_compare(ctx, a, b)
    for m in (a, b):
        mm.mm_release_map(ctx, m)
    assert st["rms_dm"] < 0.2 and st["ks_p"] > 0.997
    from oracle import stats as ostats
    ca, ta = oracle.shoot_map(dict(cfg, margin=1.5), f0)
    cb, tb = oracle.shoot_map(dict(cfg, **ORND), f0)
    assert map_l1(ca, cb) > 0
    a, b = restore(ctx, lh, cfg, ca, ta, len(f0.x)), restore(ctx, lh, cfg, cb, tb, len(f0.x))
    got = mm.mm_map_compare(ctx, a, b)
    for m in (a, b):
        mm.mm_release_map(ctx, m)
    ref = ostats.compare(ca, 4000.0, cb, 4000.0)
    assert ref["rms_dm"] < 0.2 and ref["ks_p"] > 0.997
    assert got["ks_d"] == pytest.approx(ref["ks_d"], abs=1e-15)
    assert got["rms_dm"] == pytest.approx(ref["rms_dm"], rel=1e-9)
    assert got["ks_p"] == pytest.approx(ref["ks_p"], abs=1e-6)


def test_random_maps_in_a_batch_are_identical_to_alone(ctx, f0):
    lh = mm.mm_create_lenses_from(ctx, f0.x, f0.y, f0.m)
    plist = [P(CFG0), P(CFG0, **RND), P(CFG0, ray_mode=mm.MM_RAYS_RANDOM, ray_seed=SEED + 1),
             P(CFG0, precision=mm.MM_FP64, ray_rect=(64, 64 * 9, 32, 32 * 7), **RND)]
    maps = mm.mm_shoot_batch(ctx, [lh] * len(plist), plist)
    for p, m in zip(plist, maps):
        got, st = mm.mm_map_fetch(ctx, m)
        mm.mm_release_map(ctx, m)
        alone, st1 = shoot(ctx, lh, p)
        assert np.array_equal(got, alone)
        assert (st["rays_in"], st["rays_out"]) == (st1["rays_in"], st1["rays_out"])
    a, _ = shoot(ctx, lh, plist[1])
    b, _ = shoot(ctx, lh, plist[2])
    assert not np.array_equal(a, b)                          # the seed moves the rays


def test_random_map_in_parts_equals_one_shot(ctx, f0):
    lh = mm.mm_create_lenses_from(ctx, f0.x, f0.y, f0.m)
    whole, st = shoot(ctx, lh, P(CFG0, **RND))
    g = oracle.geometry(dict(CFG0, **ORND))
    m = mm.mm_shoot(ctx, lh, P(CFG0, ray_rect=(0, 0, 0, 0), **RND))
    for r in ((0, 64 * 20, 0, g["ny"]), (64 * 20, g["nx"], 32 * 40, g["ny"]), (64 * 20, g["nx"], 0, 32 * 40)):
        mm.mm_shoot_into(ctx, 0, P(CFG0, ray_rect=r, **RND), m)
    got, st2 = mm.mm_map_fetch(ctx, m)
    assert np.array_equal(got, whole)
    assert (st2["rays_in"], st2["rays_out"]) == (st["rays_in"], st["rays_out"])
    for bad in (P(CFG0, ray_rect=(10, 64, 0, 32), **RND), P(CFG0, ray_rect=(0, 64, 0, 32))):
        with pytest.raises(mm.MMError) as e:                 # unaligned part; other ray mode than the map's
            mm.mm_shoot_into(ctx, 0, bad, m)
        assert e.value.code == mm.MM_EINVAL
    mm.mm_release_map(ctx, m)


def test_random_rays_are_refused_where_the_lattice_is_required(ctx, f0):
    lh = mm.mm_create_lenses_from(ctx, f0.x, f0.y, f0.m)
    for call in (lambda: mm.mm_submit(ctx, lh, P(CFG0, **RND)),
                 lambda: mm.mm_shoot(ctx, lh, P(CFG0, precision=mm.MM_FAR32, **RND))):
        with pytest.raises(mm.MMError) as e:
            call()
        assert e.value.code == mm.MM_EINVAL
