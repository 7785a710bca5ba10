"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances for the FP32 compensated path (rays passing very close to a lens
carry the largest FP32 error, about 6e-6 Einstein radii on these fields):
  * per-ray deflection: max |alpha_gpu - alpha_oracle| <= 1e-5 Einstein radii;
  * rays binned to a different pixel than the oracle's: <= 1e-4 of the rays;
  * maps: sum |N_gpu - N_oracle| <= 2e-4 of the rays shot (a misbinned ray
    moves at most two pixel counts);
  * ray totals exact: shot = nx * ny (or the rectangle's area) = in + out,
    and the map sums to `in`.
The plain FP64 kernel sums in the oracle's lens order; it may differ from the
oracle only by rounding, so it allows <= max(1, 1e-8 * shot) misbinned rays
and alpha within 1e-9 relative.
"""
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

CFG0 = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=4.0, npix_side=128, nrays=100.0)
CFG1 = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=20.0, npix_side=1024, nrays=2000.0)
CFG2 = dict(sigma=0.8, gamma=0.3, smooth_frac=0.5, side=40.0, npix_side=2048, nrays=500.0)


def field0():
    return synth.lens_field(100, field.radius_for_nstar(100, 0.4), 1)


def field1():
    n, r = field.nstar_rule(0.4, 0.0, 0.0, 20.0)
    return synth.lens_field(n, r, 2)


def field2():
    return synth.lens_field(25000, field.radius_for_nstar(25000, 0.4), 3)


@pytest.fixture(scope="module")
def ctx():
    mm.build()
    c = mm.mm_init(0)
    yield c
    mm.mm_destroy(c)


def lens(ctx, f):
    return mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)


def P(cfg, **kw):
    d = dict(cfg)
    d.update(kw)
    return mm.params(**d)


def shoot(ctx, lh, cfg, **kw):
    m = mm.mm_shoot(ctx, lh, P(cfg, **kw))
    counts, st = mm.mm_map_fetch(ctx, m)
    mm.mm_release_map(ctx, m)
    return counts, st


def check_totals(counts, st, shot):
    assert st["rays_shot"] == shot
    assert st["rays_in"] + st["rays_out"] == shot
    assert int(counts.sum(dtype=np.int64)) == st["rays_in"]


def map_l1(a, b):
    return int(np.abs(a.astype(np.int64) - b.astype(np.int64)).sum())


def oracle_cfg(cfg):
    return dict(cfg, margin=1.5)


def rays_check(ctx, lh, cfg, f, ii, jj, precision=mm.MM_FP32C):
    a_g, p_g = mm.mm_debug_deflect(ctx, lh, P(cfg, precision=precision), ii, jj)
    a_o, _, p_o = oracle.shoot_rays(oracle_cfg(cfg), f, ii, jj)
    err = np.hypot(a_g[:, 0] - a_o[:, 0], a_g[:, 1] - a_o[:, 1])
    mis = float(np.mean(p_g != p_o)) if len(p_g) else 0.0
    print(f"rays {len(err)}: max |d alpha| {err.max() if len(err) else 0:.3e}, mean {err.mean() if len(err) else 0:.3e}, "
          f"misbinned {mis:.3e} (precision {precision})")
    return err, mis, a_g, a_o, p_g, p_o


# ----------------------------------------------------------------- config 0 ---

def test_cfg0_fp32_full_map_matches_oracle(ctx):
    f = field0()
    lh = lens(ctx, f)
    got, st = shoot(ctx, lh, CFG0)
    ref, tot = oracle.shoot_map(oracle_cfg(CFG0), f)
    check_totals(got, st, tot["shot"])
    assert st["interactions"] == tot["shot"] * 100
    assert map_l1(got, ref) <= 2 * MISBIN_TOL * tot["shot"]
    assert abs(st["rays_in"] - tot["inside"]) <= MISBIN_TOL * tot["shot"]


def test_cfg0_fp32_every_ray_deflection_and_pixel(ctx):
    f = field0()
    lh = lens(ctx, f)
    g = oracle.geometry(oracle_cfg(CFG0))
    jj, ii = np.meshgrid(np.arange(g["ny"]), np.arange(g["nx"]), indexing="ij")
    err, mis, *_ = rays_check(ctx, lh, CFG0, f, ii.ravel(), jj.ravel())
    assert err.max() <= ALPHA_TOL, err.max()
    assert mis <= MISBIN_TOL, mis


def test_cfg0_fp64_matches_oracle(ctx):
    f = field0()
    lh = lens(ctx, f)
    got, st = shoot(ctx, lh, CFG0, precision=mm.MM_FP64)
    ref, tot = oracle.shoot_map(oracle_cfg(CFG0), f)
    check_totals(got, st, tot["shot"])
    assert map_l1(got, ref) <= 2 * max(1, 1e-8 * tot["shot"])
    rng = np.random.default_rng(0)
    g = oracle.geometry(oracle_cfg(CFG0))
    ii, jj = rng.integers(0, g["nx"], 20000), rng.integers(0, g["ny"], 20000)
    err, mis, a_g, a_o, p_g, p_o = rays_check(ctx, lh, CFG0, f, ii, jj, precision=mm.MM_FP64)
    assert np.all(np.abs(a_g - a_o) <= 1e-9 * (1 + np.abs(a_o)))
    assert np.sum(p_g != p_o) <= 1


def test_maps_are_deterministic(ctx):
    """Counts are integer atomics and every float sum has a fixed order, so repeated runs give
    the same map bit for bit: ten runs of the FP32 path, three of FP64 and of the far field."""
    f = field0()
    lh = lens(ctx, f)
    for kw, runs in ((dict(), 10), (dict(precision=mm.MM_FP64), 3), (dict(precision=mm.MM_FAR32), 3)):
        first, st0 = shoot(ctx, lh, CFG0, **kw)
        for _ in range(runs - 1):
            again, st = shoot(ctx, lh, CFG0, **kw)
            np.testing.assert_array_equal(first, again)
            assert (st["rays_in"], st["rays_out"]) == (st0["rays_in"], st0["rays_out"])


# ----------------------------------------------------------------- config 1 ---

def test_cfg1_sampled_rays(ctx):
    f = field1()
    assert f.n == 558
    lh = lens(ctx, f)
    g = oracle.geometry(oracle_cfg(CFG1))
    rng = np.random.default_rng(1)
    n = 1_000_000
    ii, jj = rng.integers(0, g["nx"], n), rng.integers(0, g["ny"], n)
    err, mis, *_ = rays_check(ctx, lh, CFG1, f, ii, jj)
    assert err.max() <= ALPHA_TOL, err.max()
    assert mis <= MISBIN_TOL, mis


def test_cfg1_full_map_totals_and_window_parity(ctx):
    f = field1()
    lh = lens(ctx, f)
    g = oracle.geometry(oracle_cfg(CFG1))
    got, st = shoot(ctx, lh, CFG1)
    check_totals(got, st, g["nx"] * g["ny"])
    assert st["interactions"] == g["nx"] * g["ny"] * 558
    # mean magnification of the full map is close to the theoretical one (weak check)
    assert abs(st["mu_mean"] / field.mu_theory(0.4, 0.0) - 1) < 0.1
    # a window of 2048^2 rays (ragged: not a multiple of the tile) against the oracle
    c = g["nx"] // 2
    rect = (c - 1000, c + 1049, c - 700, c + 1349)
    gw, sw = shoot(ctx, lh, CFG1, ray_rect=rect)
    ref, tot = oracle.shoot_map(oracle_cfg(CFG1), f, rect=rect)
    check_totals(gw, sw, tot["shot"])
    assert map_l1(gw, ref) <= 2 * MISBIN_TOL * tot["shot"]


# ----------------------------------------------------------------- config 2 ---

def test_cfg2_sampled_rays_and_window(ctx):
    """Config 2 (sigma = 0.8, s = 0.5, gamma = 0.3, N* = 25000): 10^6 rays sampled over the whole
    686921 x 137385-ray grid against the oracle, and a ragged 601 x 450-ray window map."""
    f = field2()
    lh = lens(ctx, f)
    g = oracle.geometry(oracle_cfg(CFG2))
    rng = np.random.default_rng(2)
    n = 1_000_000
    ii, jj = rng.integers(0, g["nx"], n), rng.integers(0, g["ny"], n)
    err, mis, *_ = rays_check(ctx, lh, CFG2, f, ii, jj)
    assert err.max() <= ALPHA_TOL, err.max()
    assert mis <= MISBIN_TOL, mis
    ci, cj = g["nx"] // 2, g["ny"] // 2
    rect = (ci - 300, ci + 301, cj - 200, cj + 250)
    gw, sw = shoot(ctx, lh, CFG2, ray_rect=rect)
    ref, tot = oracle.shoot_map(oracle_cfg(CFG2), f, rect=rect)
    check_totals(gw, sw, tot["shot"])
    assert map_l1(gw, ref) <= 2 * max(2, MISBIN_TOL * tot["shot"])


def central_window_rect(g, cfg, window_px=256, margin=1.5):
    """Rays of the global grid that the mean lens equation, y = diag(1-sigma-gamma, 1-sigma+gamma) x,
    maps into the central window_px^2 pixels, widened by `margin` per side (Eq. square applied to
    the window): [i0, i1) x [j0, j1)."""
    a = abs(1 - cfg["sigma"] - cfg["gamma"])
    b = abs(1 - cfg["sigma"] + cfg["gamma"])
    hs = 0.5 * window_px * g["pix"]
    hx, hy = margin * hs / a, margin * hs / b
    d = g["delta"]
    i0 = max(0, int(np.floor(-hx / d + g["nx"] / 2))); i1 = min(g["nx"], int(np.ceil(hx / d + g["nx"] / 2)))
    j0 = max(0, int(np.floor(-hy / d + g["ny"] / 2))); j1 = min(g["ny"], int(np.ceil(hy / d + g["ny"] / 2)))
    return i0, i1, j0, j1


def test_cfg2_central_window_error_report(ctx):
    """Error report of config 2 on the rays that map back to the central 256^2-pixel window (x 1.5):
    a 75 x 15 Einstein-radius region of 1.47e9 rays. The FP32 map of the whole window is shot
    (totals exact); every 16th ray row and column of it (5.8e6 rays) is computed by the oracle,
    by the FP32 kernel (through the map kernel's code) and by the plain FP64 kernel, and for each
    GPU form the report gives the max and mean |d alpha| (Einstein radii), the fraction of rays
    binned to another pixel, and the L1 distance of the strided maps over the rays shot. Bars:
    FP32 max |d alpha| <= 1e-5, misbinned <= 1e-4, L1 <= 2e-4; FP64 alpha within 1e-9 relative,
    misbinned <= max(1, 1e-8 n) rays."""
    import json
    f = field2()
    lh = lens(ctx, f)
    g = oracle.geometry(oracle_cfg(CFG2))
    rect = central_window_rect(g, CFG2)
    assert 85000 <= rect[1] - rect[0] <= 87000 and 17000 <= rect[3] - rect[2] <= 17400
    gw, sw = shoot(ctx, lh, CFG2, ray_rect=rect)
    check_totals(gw, sw, (rect[1] - rect[0]) * (rect[3] - rect[2]))
    stride = 16
    jj, ii = np.meshgrid(np.arange(rect[2], rect[3], stride), np.arange(rect[0], rect[1], stride), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    n = ii.size
    a_o, _, p_o = oracle.shoot_rays(oracle_cfg(CFG2), f, ii, jj)
    nside = CFG2["npix_side"]
    map_o = np.bincount(p_o[p_o >= 0], minlength=nside * nside)
    report = {"workload": "config 2, central 256^2-pixel window x 1.5 (rays " + str(rect) + f"), every {stride}th "
                          f"ray row and column: {n} rays x {f.n} lenses",
              "window_map_fp32": {"rays_shot": sw["rays_shot"], "rays_in": sw["rays_in"], "rays_out": sw["rays_out"]}}
    for name, prec in (("fp32", mm.MM_FP32C), ("fp64", mm.MM_FP64)):
        a_g, p_g = mm.mm_debug_deflect(ctx, lh, P(CFG2, precision=prec), ii, jj)
        err = np.hypot(a_g[:, 0] - a_o[:, 0], a_g[:, 1] - a_o[:, 1])
        mis = int(np.sum(p_g != p_o))
        map_g = np.bincount(p_g[p_g >= 0], minlength=nside * nside)
        l1 = int(np.abs(map_g - map_o).sum())
        report[name] = {"max_dalpha_re": float(err.max()), "mean_dalpha_re": float(err.mean()),
                        "misbinned_fraction": mis / n, "strided_map_l1_over_rays": l1 / n,
                        "max_rel_dalpha": float(np.max(np.abs(a_g - a_o) / (1 + np.abs(a_o))))}
        if prec == mm.MM_FP32C:
            assert err.max() <= ALPHA_TOL, err.max()
            assert mis <= MISBIN_TOL * n, mis
            assert l1 <= 2 * MISBIN_TOL * n, l1
        else:
            assert np.all(np.abs(a_g - a_o) <= 1e-9 * (1 + np.abs(a_o)))
            assert mis <= max(1, 1e-8 * n), mis
    print("CFG2_WINDOW_REPORT " + json.dumps(report))


def test_fp64_ray_list_equals_the_fp64_map_kernel(ctx):
    """Per-ray FP64 results (mm_debug_deflect, one thread per listed ray) equal the FP64 map kernel's:
    every ray of a ragged sheared window, binned on the host, gives the map bit for bit."""
    cfg = dict(sigma=0.6, gamma=0.25, smooth_frac=0.3, side=3.0, npix_side=48, nrays=36.0)
    f = synth.lens_field(777, 14.0, 12, synth.MASS_LOGNORMAL)
    lh = lens(ctx, f)
    g = oracle.geometry(oracle_cfg(cfg))
    rect = (g["nx"] // 2 - 211, g["nx"] // 2 + 190, g["ny"] // 2 - 95, g["ny"] // 2 + 70)
    got, st = shoot(ctx, lh, cfg, ray_rect=rect, precision=mm.MM_FP64)
    jj, ii = np.meshgrid(np.arange(rect[2], rect[3]), np.arange(rect[0], rect[1]), indexing="ij")
    _, pix = mm.mm_debug_deflect(ctx, lh, P(cfg, precision=mm.MM_FP64), ii.ravel(), jj.ravel())
    inside = pix[pix >= 0]
    np.testing.assert_array_equal(np.bincount(inside, minlength=48 * 48).reshape(48, 48), got)
    assert (inside.size, int(np.sum(pix < 0))) == (st["rays_in"], st["rays_out"])
    mm.mm_release_lenses(ctx, lh)


# -------------------------------------------------------- lognormal masses ---

def mix_windows(count=4, seed=4):
    out = []
    for d in synth.map_mix(count, seed):
        cfg = dict(sigma=d.sigma, gamma=d.gamma, smooth_frac=d.smooth_frac, side=d.side, npix_side=d.npix_side,
                   nrays=d.nrays)
        mmean = field.mean_mass(1, 0.0, 0.5)
        n, r = field.nstar_rule(d.sigma, d.gamma, d.smooth_frac, d.side, 1.5, mmean)
        n = min(n, 20000)
        f = synth.lens_field(n, r, d.seed, synth.MASS_LOGNORMAL, 0.0, 0.5)
        g = oracle.geometry(oracle_cfg(cfg))
        ci, cj = g["nx"] // 2, g["ny"] // 2
        rect = (max(0, ci - 200), min(g["nx"], ci + 233), max(0, cj - 150), min(g["ny"], cj + 170))
        out.append((cfg, f, rect))
    return out


def test_lognormal_mix_windows_match_oracle(ctx):
    for cfg, f, rect in mix_windows():
        lh = lens(ctx, f)
        gw, sw = shoot(ctx, lh, cfg, ray_rect=rect)
        ref, tot = oracle.shoot_map(oracle_cfg(cfg), f, rect=rect)
        check_totals(gw, sw, tot["shot"])
        assert map_l1(gw, ref) <= 2 * max(2, MISBIN_TOL * tot["shot"]), cfg
        ii = np.arange(rect[0], rect[1], 7)
        jj = np.full(ii.shape, (rect[2] + rect[3]) // 2)
        err, mis, *_ = rays_check(ctx, lh, cfg, f, ii, jj)
        assert err.max() <= ALPHA_TOL, (cfg, err.max())
        mm.mm_release_lenses(ctx, lh)


@pytest.mark.parametrize("spectrum", ["lognormal", "light", "wide", "with_zeros"])
def test_mass_spectra_match_oracle(ctx, spectrum):
    """The FP32 path with mass spectra other than unit masses: lognormal masses, the same
    times 1/256, log-uniform masses spanning five decades, and lognormal masses with
    every seventh lens of zero mass."""
    cfg = dict(sigma=0.5, gamma=0.2, smooth_frac=0.2, side=4.0, npix_side=64, nrays=64.0)
    f0 = synth.lens_field(700, 12.0, 31, synth.MASS_LOGNORMAL)
    m = f0.m.copy()
    if spectrum == "light":
        m = m / 256.0
    elif spectrum == "wide":
        m = 10.0 ** np.random.default_rng(31).uniform(-4.0, 1.0, len(m))
    elif spectrum == "with_zeros":
        m[::7] = 0.0
    f = synth.LensField(f0.x, f0.y, m)
    g = oracle.geometry(oracle_cfg(cfg))
    rect = (g["nx"] // 2 - 160, g["nx"] // 2 + 150, g["ny"] // 2 - 100, g["ny"] // 2 + 90)
    lh = lens(ctx, f)
    got, st = shoot(ctx, lh, cfg, ray_rect=rect)
    ref, tot = oracle.shoot_map(oracle_cfg(cfg), f, rect=rect)
    check_totals(got, st, tot["shot"])
    assert map_l1(got, ref) <= 2 * max(2, MISBIN_TOL * tot["shot"]), spectrum
    jj, ii = np.meshgrid(np.arange(rect[2], rect[3], 3), np.arange(rect[0], rect[1], 5), indexing="ij")
    err, mis, *_ = rays_check(ctx, lh, cfg, f, ii.ravel(), jj.ravel())
    assert err.max() <= ALPHA_TOL, (spectrum, err.max())
    assert mis <= MISBIN_TOL
    mm.mm_release_lenses(ctx, lh)


# ------------------------------------------------------------- edge cases ---

def test_smooth_only_map_exact(ctx):
    """N* = 0, all matter smooth: the FP32 epilogue must reproduce the oracle's exact integer map."""
    cfg = dict(sigma=0.53, gamma=0.1, smooth_frac=1.0, side=2.0, npix_side=16, nrays=121.0)
    empty = synth.lens_field(0, 1.0, 0)
    lh = lens(ctx, empty)
    got, st = shoot(ctx, lh, cfg)
    ref, tot = oracle.shoot_map(oracle_cfg(cfg), empty)
    np.testing.assert_array_equal(got, ref)
    check_totals(got, st, tot["shot"])
    got64, _ = shoot(ctx, lh, cfg, precision=mm.MM_FP64)
    np.testing.assert_array_equal(got64, ref)


def test_single_lens_and_ray_on_lens(ctx):
    cfg = dict(sigma=0.0, gamma=0.0, smooth_frac=0.0, side=2.0, npix_side=16, nrays=16.0)
    g = oracle.geometry(oracle_cfg(cfg))
    x1 = (3 + 0.5 - 0.5 * g["nx"]) * g["delta"]
    x2 = (5 + 0.5 - 0.5 * g["ny"]) * g["delta"]
    f = synth.LensField(np.array([x1]), np.array([x2]), np.array([1.0]))
    lh = lens(ctx, f)
    for prec in (mm.MM_FP32C, mm.MM_FP64):
        _, pix = mm.mm_debug_deflect(ctx, lh, P(cfg, precision=prec), [3], [5])
        assert pix[0] == -1
        got, st = shoot(ctx, lh, cfg, precision=prec)
        ref, tot = oracle.shoot_map(oracle_cfg(cfg), f)
        check_totals(got, st, tot["shot"])
        assert map_l1(got, ref) <= 2


def test_empty_and_tiny_rectangles(ctx):
    f = field0()
    lh = lens(ctx, f)
    got, st = shoot(ctx, lh, CFG0, ray_rect=(10, 10, 0, 5))
    assert st["rays_shot"] == 0 and got.sum() == 0
    got, st = shoot(ctx, lh, CFG0, ray_rect=(1600, 1601, 1700, 1701))
    ref, tot = oracle.shoot_map(oracle_cfg(CFG0), f, rect=(1600, 1601, 1700, 1701))
    check_totals(got, st, 1)
    np.testing.assert_array_equal(got, ref)


def test_odd_lens_counts_around_chunk_boundaries(ctx):
    cfg = dict(sigma=0.4, gamma=0.1, smooth_frac=0.2, side=8.0, npix_side=256, nrays=9.0)
    g = oracle.geometry(oracle_cfg(cfg))
    rect = (g["nx"] // 2 - 150, g["nx"] // 2 + 150, g["ny"] // 2 - 100, g["ny"] // 2 + 100)
    for n in (1, 2, 3, 511, 512, 513, 1025):
        f = synth.lens_field(n, 12.0, 100 + n)
        lh = lens(ctx, f)
        got, st = shoot(ctx, lh, cfg, ray_rect=rect)
        ref, tot = oracle.shoot_map(oracle_cfg(cfg), f, rect=rect)
        check_totals(got, st, tot["shot"])
        assert map_l1(got, ref) <= 2 * max(2, MISBIN_TOL * tot["shot"]), n
        mm.mm_release_lenses(ctx, lh)


def test_maximum_map_side(ctx):
    """N_side = 32768, the largest map: flat pixel indices up to 2^30 agree with the oracle."""
    cfg = dict(sigma=0.4, gamma=0.1, smooth_frac=0.2, side=8.0, npix_side=32768, nrays=0.01)
    f = synth.lens_field(200, 10.0, 77)
    lh = lens(ctx, f)
    g = oracle.geometry(oracle_cfg(cfg))
    rng = np.random.default_rng(3)
    ii, jj = rng.integers(0, g["nx"], 50_000), rng.integers(0, g["ny"], 50_000)
    err, mis, a_g, a_o, p_g, p_o = rays_check(ctx, lh, cfg, f, ii, jj)
    assert err.max() <= ALPHA_TOL
    # pixels here are 80x smaller than in the configs (p = 2.4e-4 Einstein radii), and a
    # ray is misbinned with probability ~ 2 |d alpha| / p: bound it by the measured mean
    # deflection error, and require every mismatch to be a neighbouring pixel
    assert mis <= max(MISBIN_TOL, 4.0 * err.mean() / (8.0 / 32768)), (mis, err.mean())
    bad = (p_g != p_o) & (p_g >= 0) & (p_o >= 0)
    assert np.all(np.abs(p_g[bad] % 32768 - p_o[bad] % 32768) <= 1)
    assert np.all(np.abs(p_g[bad] // 32768 - p_o[bad] // 32768) <= 1)
    assert p_o.max() > 2 ** 29
    m = mm.mm_shoot(ctx, lh, P(cfg))
    _, st = mm.mm_map_fetch(ctx, m, want_counts=False)
    assert st["rays_shot"] == g["nx"] * g["ny"] == st["rays_in"] + st["rays_out"]
    mm.mm_release_map(ctx, m)


def test_every_variant_within_tolerance(ctx):
    f = field1()
    lh = lens(ctx, f)
    g = oracle.geometry(oracle_cfg(CFG1))
    rng = np.random.default_rng(7)
    ii, jj = rng.integers(0, g["nx"], 100_000), rng.integers(0, g["ny"], 100_000)
    try:
        for v in range(mm.mm_variant_count()):
            mm.mm_set_variant(ctx, v)
            err, mis, *_ = rays_check(ctx, lh, CFG1, f, ii, jj)
            assert err.max() <= ALPHA_TOL and mis <= MISBIN_TOL, (v, err.max(), mis)
    finally:
        mm.mm_set_variant(ctx, -1)


def test_split_tiles_match_oracle(ctx):
    """A window of the N* = 25 000 map has ~150 tiles: each tile's lens sum is split over several
    CTAs and recombined; maps, deflections and pixels must still match the oracle."""
    f = field2()
    lh = lens(ctx, f)
    g = oracle.geometry(oracle_cfg(CFG2))
    rect = (g["nx"] // 3, g["nx"] // 3 + 577, g["ny"] // 2, g["ny"] // 2 + 389)
    m = mm.mm_shoot(ctx, lh, P(CFG2, ray_rect=rect))
    got, st = mm.mm_map_fetch(ctx, m)
    mm.mm_release_map(ctx, m)
    assert st["lens_splits"] > 1
    ref, tot = oracle.shoot_map(oracle_cfg(CFG2), f, rect=rect)
    check_totals(got, st, tot["shot"])
    assert map_l1(got, ref) <= 2 * max(2, MISBIN_TOL * tot["shot"])
    rng = np.random.default_rng(9)
    ii = rng.integers(rect[0], rect[1], 4000)
    jj = rng.integers(rect[2], rect[3], 4000)
    a_g, p_g = mm.mm_debug_deflect(ctx, lh, P(CFG2, ray_rect=rect), ii, jj)
    a_o, _, p_o = oracle.shoot_rays(oracle_cfg(CFG2), f, ii, jj)
    err = np.hypot(a_g[:, 0] - a_o[:, 0], a_g[:, 1] - a_o[:, 1])
    assert err.max() <= ALPHA_TOL and np.mean(p_g != p_o) <= MISBIN_TOL
    # the whole-grid map of the same field has millions of tiles: no split
    m = mm.mm_shoot(ctx, lh, P(CFG2, ray_rect=(0, 64 * 200, 0, 32 * 200)))
    _, st = mm.mm_map_fetch(ctx, m, want_counts=False)
    mm.mm_release_map(ctx, m)
    assert st["lens_splits"] == 1


def test_thread_layouts_give_bit_identical_maps(ctx):
    """Every thread layout runs the same per-ray FP32 operations on the same tiles."""
    items = mix_windows(2, 21)
    cases = [(CFG1, field1(), (50000, 50700, 50000, 50300))] + items
    try:
        for cfg, f, rect in cases:
            lh = lens(ctx, f)
            maps = []
            for lay in range(mm.mm_layout_count()):
                mm.mm_set_layout(ctx, lay)
                maps.append(shoot(ctx, lh, cfg, ray_rect=rect)[0])
                a, p = mm.mm_debug_deflect(ctx, lh, P(cfg), [rect[0] + 5, rect[0] + 77], [rect[2] + 3, rect[2] + 40])
                if lay == 0:
                    a0, p0 = a, p
                np.testing.assert_array_equal(a, a0)
                np.testing.assert_array_equal(p, p0)
            for m in maps[1:]:
                np.testing.assert_array_equal(m, maps[0])
    finally:
        mm.mm_set_layout(ctx, 1)


# ---------------------------------------------- lens sets, batch, serving ---

def test_library_lens_generator_matches_input_module(ctx):
    for cfg, seed, model in ((CFG1, 2, 0), (dict(CFG2, nstar=3000), 9, 1)):
        p = P(cfg, seed=seed, mass_model=model)
        h = mm.mm_create_lenses(ctx, p)
        x, y, m = mm.mm_lenses_fetch(ctx, h)
        geo = mm.mm_geometry_of(p)
        ref = synth.lens_field(geo["nstar"], geo["disc_radius"], seed, model, 0.0, 0.5)
        np.testing.assert_array_equal(x, ref.x)
        np.testing.assert_array_equal(y, ref.y)
        np.testing.assert_allclose(m, ref.m, rtol=1e-14)


def test_batch_results_identical_to_alone(ctx):
    items = mix_windows(6, 11)
    plist, hl, alone = [], [], []
    for cfg, f, rect in items:
        h = lens(ctx, f)
        hl.append(h)
        plist.append(P(cfg, ray_rect=rect))
        alone.append(shoot(ctx, h, cfg, ray_rect=rect)[0])
    maps = mm.mm_shoot_batch(ctx, hl, plist)
    for m, a in zip(maps, alone):
        got, _ = mm.mm_map_fetch(ctx, m)
        np.testing.assert_array_equal(got, a)
        mm.mm_release_map(ctx, m)


def large_request():
    """A "large" request of the served mix: 2048^2 pixels and N* = 20000 lognormal lenses with
    kappa_* = sigma_* (disc radius from Eq. nstar), here at N_rays = 4 (3.4e8 rays)."""
    cfg = dict(sigma=0.45, gamma=0.2, smooth_frac=0.3, side=20.0, npix_side=2048, nrays=4.0)
    mmean = field.mean_mass(1, 0.0, 0.5)
    f = synth.lens_field(20000, field.radius_for_nstar(20000, 0.45 * 0.7, mmean), 77, synth.MASS_LOGNORMAL)
    return cfg, f, None


@pytest.mark.parametrize("priority", [0.8, 0.0, 1.0])
def test_serving_results_identical_to_alone(ctx, priority):
    """Eight mixed-shape windows and one large whole map, served together through continuous
    batching, each equal bit for bit to the same map shot alone."""
    items = mix_windows(8, 12) + [large_request()]
    mm.mm_serve_config(ctx, max_active=4, wave_ms=0.5)
    mm.mm_serve_priority(ctx, priority)
    try:
        reqs, alone = [], []
        for k, (cfg, f, rect) in enumerate(items):
            h = lens(ctx, f)
            alone.append(shoot(ctx, h, cfg, ray_rect=rect)[0])
            reqs.append(mm.mm_submit(ctx, h, P(cfg, ray_rect=rect)))
        for r, a in zip(reqs, alone):
            m = mm.mm_wait(ctx, r, timeout_s=120)
            got, st = mm.mm_map_fetch(ctx, m)
            np.testing.assert_array_equal(got, a)
            q, t = mm.mm_req_times(ctx, r)
            assert 0 <= q <= t
            mm.mm_release_map(ctx, m)
    finally:
        mm.mm_serve_priority(ctx, 0.8)


def test_serving_small_request_overtakes_a_large_one(ctx):
    """Shortest remaining work first: a small map submitted just after a large one
    finishes first, and the large one still finishes (every map moves each wave)."""
    mm.mm_serve_config(ctx, max_active=8, wave_ms=0.5)
    mm.mm_serve_priority(ctx, 1.0)
    try:
        big = mm.mm_submit(ctx, 0, P(CFG1, nstar=558, seed=2, ray_rect=(0, 16384, 0, 8192)))   # 7.5e10
        small = mm.mm_submit(ctx, 0, P(CFG0, nstar=100, seed=1, ray_rect=(0, 640, 0, 640)))    # 4.1e7
        ms = mm.mm_wait(ctx, small, timeout_s=120)
        mb = mm.mm_wait(ctx, big, timeout_s=120)
        _, tsmall = mm.mm_req_times(ctx, small)
        _, tbig = mm.mm_req_times(ctx, big)
        assert tsmall < tbig
        _, st = mm.mm_map_fetch(ctx, mb, want_counts=False)
        assert st["rays_shot"] == 16384 * 8192 == st["rays_in"] + st["rays_out"]
        mm.mm_release_map(ctx, ms)
        mm.mm_release_map(ctx, mb)
    finally:
        mm.mm_serve_priority(ctx, 0.8)


def test_serving_cancels_an_admitted_request(ctx):
    """An admitted request cancelled in mid-map stops at the next wave and reports MM_ECANCELED; the
    counters account for it, and the server goes on serving (a later request equals its map alone)."""
    mm.mm_serve_config(ctx, max_active=4, wave_ms=0.5)
    before = mm.mm_serve_stats(ctx)
    f = field1()
    lh = lens(ctx, f)
    big = mm.mm_submit(ctx, lh, P(CFG1))                 # the Fig. 1 map, 7.3e12 interactions
    import time
    time.sleep(0.3)
    mm.mm_cancel(ctx, big)
    with pytest.raises(mm.MMError) as e:
        mm.mm_wait(ctx, big, timeout_s=60)
    assert e.value.code == mm.MM_ECANCELED
    with pytest.raises(mm.MMError) as e2:                 # ended: nothing left to cancel
        mm.mm_cancel(ctx, big)
    assert e2.value.code == mm.MM_EBUSY
    after = mm.mm_serve_stats(ctx)
    assert after["cancelled"] == before["cancelled"] + 1
    shot = after["interactions"] - before["interactions"]
    assert 0 < shot < 0.9 * 7.31e12
    assert after["active"] == 0 and after["queued"] == 0
    cfg = dict(CFG0)
    r = mm.mm_submit(ctx, 0, P(cfg, nstar=100, seed=1))
    m = mm.mm_wait(ctx, r, timeout_s=60)
    got, _ = mm.mm_map_fetch(ctx, m)
    h = mm.mm_create_lenses(ctx, P(cfg, nstar=100, seed=1))
    ref, _ = shoot(ctx, h, cfg)
    np.testing.assert_array_equal(got, ref)
    done = mm.mm_serve_stats(ctx)
    assert done["completed"] == after["completed"] + 1 and done["waves"] > after["waves"]
    mm.mm_release_map(ctx, m)


def test_serving_generates_fields_and_polls(ctx):
    cfg = dict(CFG0)
    r = mm.mm_submit(ctx, 0, P(cfg, nstar=100, seed=1))
    for _ in range(20000):
        done, m = mm.mm_poll(ctx, r)
        if done:
            break
    else:
        m = mm.mm_wait(ctx, r, timeout_s=60)
    got, st = mm.mm_map_fetch(ctx, m)
    h = mm.mm_create_lenses(ctx, P(cfg, nstar=100, seed=1))
    ref, _ = shoot(ctx, h, cfg)
    np.testing.assert_array_equal(got, ref)


def test_admission_rejects_oversized_request_and_cancel():
    mm.build()
    c = mm.mm_init(0, hbm_budget_bytes=64 << 20)
    try:
        with pytest.raises(mm.MMError) as e:
            mm.mm_submit(c, 0, P(CFG1, npix_side=8192))    # 256 MiB map > 64 MiB budget
        assert e.value.code == mm.MM_ENOMEM
        mm.mm_serve_config(c, max_active=1, wave_ms=0.5)
        big = mm.mm_submit(c, 0, P(CFG1))
        small = mm.mm_submit(c, 0, P(CFG0, nstar=100))
        try:
            mm.mm_cancel(c, small)
            with pytest.raises(mm.MMError) as e2:
                mm.mm_wait(c, small, timeout_s=10)
            assert e2.value.code == mm.MM_ECANCELED
        except mm.MMError as e3:                            # already admitted: cancel refuses
            assert e3.code == mm.MM_EBUSY
        with pytest.raises(mm.MMError) as e4:
            mm.mm_wait(c, big, timeout_s=0.0)
        assert e4.value.code in (mm.MM_ETIMEDOUT,)
    finally:
        mm.mm_destroy(c)


def test_unknown_handles(ctx):
    with pytest.raises(mm.MMError) as e:
        mm.mm_shoot(ctx, 987654321, P(CFG0))
    assert e.value.code == mm.MM_ENOTFOUND
    with pytest.raises(mm.MMError):
        mm.mm_map_fetch(ctx, 987654321)
    with pytest.raises(mm.MMError):
        mm.mm_release_lenses(ctx, 987654321)


def test_large_lens_count_streams_through_chunks(ctx):
    """N* = 200 000 (391 lens chunks per tile): lenses are streamed through shared memory, so
    N* is bounded by device memory only. A ray window matches the oracle, and the far field's
    sampled rays match the far-field oracle."""
    nstar = 200000
    f = synth.lens_field(nstar, float(np.sqrt(nstar / 0.4)), 21)
    lh = lens(ctx, f)
    cfg = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=4.0, npix_side=64, nrays=50.0)
    g = mm.mm_geometry_of(P(cfg))
    c = g["nx"] // 2
    rect = (c - 160, c + 160, c - 96, c + 96)                  # 61 440 rays: 1.2e10 interactions
    got, st = shoot(ctx, lh, cfg, ray_rect=rect)
    ref, tot = oracle.shoot_map(oracle_cfg(cfg), f, rect=rect)
    assert st["rays_shot"] == tot["shot"] and st["nstar"] == nstar
    check_totals(got, st, tot["shot"])
    assert int(np.abs(got.astype(np.int64) - ref).sum()) <= max(2, 2e-4 * tot["shot"])
    rng = np.random.default_rng(21)
    ii, jj = rng.integers(0, g["nx"], 300), rng.integers(0, g["ny"], 300)
    far = dict(order=10, ratio=0.15, block_tiles=8)
    a_g, _ = mm.mm_debug_deflect(ctx, lh, P(cfg, precision=mm.MM_FAR32, far_order=far["order"],
                                           far_ratio=far["ratio"], far_block=far["block_tiles"],
                                           far_group_order=0), ii, jj)
    a_o, _, _, _ = oracle.far_rays(oracle_cfg(cfg), f, far, ii, jj)
    assert np.hypot(*(a_g - a_o).T).max() <= 1e-5


def test_serving_stress_mixed_precisions_with_cancellations(ctx):
    """96 requests of FP32, FP64 and far-field maps of varied shape submitted at once to a server
    of 5 slots, every 7th cancelled right away (if still queued). Every request ends exactly once:
    cancelled before it ran, or done with exact totals; a sample equals the same map shot alone."""
    mm.mm_serve_config(ctx, max_active=5, wave_ms=1.0)
    f = synth.lens_field(200, 10.0, 31, model=synth.MASS_LOGNORMAL)
    lh = lens(ctx, f)
    kinds = [dict(), dict(precision=mm.MM_FP64), dict(precision=mm.MM_FAR32)]
    rng = np.random.default_rng(5)
    reqs = []
    for k in range(96):
        sigma = float(rng.uniform(0.2, 0.55))
        cfg = dict(sigma=sigma, gamma=float(rng.uniform(0.0, 0.25)), smooth_frac=float(rng.uniform(0.0, 0.5)),
                   side=3.0, npix_side=int(rng.choice([32, 48, 64])), nrays=float(rng.choice([10.0, 20.0])))
        p = P(cfg, **kinds[k % 3])
        r = mm.mm_submit(ctx, lh, p)
        cancelled = False
        if k % 7 == 3:
            try:
                mm.mm_cancel(ctx, r)
                cancelled = True
            except mm.MMError as e:                      # already admitted: it runs to completion
                assert e.code == mm.MM_EBUSY
        reqs.append((r, p, cancelled))
    assert any(c for _, _, c in reqs)
    for k, (r, p, cancelled) in enumerate(reqs):
        if cancelled:
            with pytest.raises(mm.MMError) as e:
                mm.mm_wait(ctx, r, timeout_s=60)
            assert e.value.code == mm.MM_ECANCELED
            continue
        m = mm.mm_wait(ctx, r, timeout_s=300)
        got, st = mm.mm_map_fetch(ctx, m)
        check_totals(got, st, st["nx"] * st["ny"])
        mm.mm_release_map(ctx, m)
        if k % 8 == 0:
            a = mm.mm_shoot(ctx, lh, p)
            alone, _ = mm.mm_map_fetch(ctx, a)
            mm.mm_release_map(ctx, a)
            np.testing.assert_array_equal(got, alone)
