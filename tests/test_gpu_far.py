"""MM_FAR32, the far-field approximation (the tree code's idea on blocks of rays,
Sect. 2.1, Eq. hierarchical), against the oracle's statement of the same
approximation (oracle.far_rays / oracle.far_map), and against the exact method.

The GPU and the oracle compute the same approximation, so they agree to FP32
accuracy. Per ray the bar is |alpha_GPU - alpha_oracle| <= 1e-5 R_E, the exact
path's target. Maps may differ only by rays whose source position lies within
the FP32 error of a pixel edge, so the bar is 2e-4 of the rays. The tail bound
the GPU reports is the oracle's, up to FP32 rounding."""
import numpy as np
import pytest

import oracle
import paper_1005_5198_gb300 as mm
import synth
from oracle import field

pytestmark = pytest.mark.gpu

CFG0 = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=4.0, npix_side=128, nrays=100.0)
CFG1 = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=20.0, npix_side=1024, nrays=2000.0)
CFG2 = dict(sigma=0.8, gamma=0.3, smooth_frac=0.5, side=40.0, npix_side=2048, nrays=500.0)
FAR_DEFAULT = dict(order=10, ratio=0.15, block_tiles=8)     # the library's defaults
ALPHA_TOL = 1e-5
MISBIN = 2e-4


@pytest.fixture(scope="module")
def ctx():
    mm.build()
    c = mm.mm_init(0)
    yield c
    mm.mm_destroy(c)


def P(cfg, far, **kw):
    """Far-field parameters of the oracle's statement `far` (no grouping unless it says so)."""
    d = dict(cfg, precision=mm.MM_FAR32, far_order=far["order"], far_ratio=far["ratio"],
             far_block=far["block_tiles"], far_group_order=far.get("group_order", 0),
             far_group_theta=far.get("group_theta", 0.5), far_group_leaf=far.get("group_leaf", 64))
    d.update(kw)
    return mm.params(**d)


def ocfg(cfg):
    return dict(cfg, margin=1.5)


def field0():
    return synth.lens_field(100, field.radius_for_nstar(100, 0.4), 1)


def sample_rays(nx, ny, n, seed, rect=None):
    rng = np.random.default_rng(seed)
    i0, i1, j0, j1 = rect if rect is not None else (0, nx, 0, ny)
    return rng.integers(i0, i1, n), rng.integers(j0, j1, n)


def check_rays(ctx, lh, f, cfg, far, ii, jj, rect=None):
    kw = {} if rect is None else dict(ray_rect=rect)
    a_g, p_g = mm.mm_debug_deflect(ctx, lh, P(cfg, far, **kw), ii, jj)
    origin = (0, 0) if rect is None else (rect[0], rect[2])
    a_o, y_o, p_o, b_o = oracle.far_rays(ocfg(cfg), f, far, ii, jj, origin=origin)
    err = np.hypot(*(a_g - a_o).T)
    assert err.max() <= ALPHA_TOL, f"max |d alpha| = {err.max():.3g}"
    # pixels differ only where the oracle's source position is within the error of an edge
    bad = p_g != p_o
    if bad.any():
        pix = cfg["side"] / cfg["npix_side"]
        u = (y_o[bad] + cfg["side"] / 2) / pix
        edge = np.abs(u - np.round(u)).min(axis=1) * pix
        assert np.all(edge <= 4 * err[bad] + 1e-9), "a pixel mismatch away from a pixel edge"
    assert bad.mean() <= MISBIN
    return err, b_o


@pytest.mark.parametrize("far", [FAR_DEFAULT, dict(order=4, ratio=0.5, block_tiles=4),
                                 dict(order=1, ratio=0.2, block_tiles=2), dict(order=32, ratio=0.6, block_tiles=16),
                                 dict(order=9, ratio=0.45, block_tiles=3)],
                         ids=["default", "P4", "P1", "P32", "P9-bt3"])
def test_rays_match_the_oracle_config0(ctx, far):
    f = field0()
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    g = mm.mm_geometry_of(mm.params(**CFG0))
    ii, jj = sample_rays(g["nx"], g["ny"], 20000, 1)
    check_rays(ctx, lh, f, CFG0, far, ii, jj)
    mm.mm_release_lenses(ctx, lh)


def test_map_matches_the_oracle_and_the_bound_config0(ctx):
    f = field0()
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    for far in (FAR_DEFAULT, dict(order=6, ratio=0.5, block_tiles=4)):
        m = mm.mm_shoot(ctx, lh, P(CFG0, far))
        got, st = mm.mm_map_fetch(ctx, m)
        mm.mm_release_map(ctx, m)
        ref, tot, bmax = oracle.far_map(ocfg(CFG0), f, far)
        assert st["rays_shot"] == tot["shot"] and st["rays_in"] + st["rays_out"] == st["rays_shot"]
        assert int(got.sum()) == st["rays_in"]
        assert int(np.abs(got.astype(np.int64) - ref).sum()) <= 2 * MISBIN * tot["shot"]
        assert st["far_bound"] == pytest.approx(bmax, rel=2e-3)
    mm.mm_release_lenses(ctx, lh)


def test_every_lens_near_is_the_exact_method(ctx):
    f = field0()
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    far = dict(order=8, ratio=1e-6, block_tiles=8)             # rho / q covers the whole field
    m = mm.mm_shoot(ctx, lh, P(CFG0, far))
    got, st = mm.mm_map_fetch(ctx, m)
    mm.mm_release_map(ctx, m)
    ref, tot = oracle.shoot_map(ocfg(CFG0), f)                  # the exact method's oracle
    assert st["far_bound"] == 0.0 and st["rays_shot"] == tot["shot"]
    assert int(np.abs(got.astype(np.int64) - ref).sum()) <= 2 * MISBIN * tot["shot"]
    mm.mm_release_lenses(ctx, lh)


def test_ragged_window_with_lognormal_masses(ctx):
    f = synth.lens_field(300, 12.0, 7, model=synth.MASS_LOGNORMAL)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    cfg = dict(sigma=0.55, gamma=0.2, smooth_frac=0.3, side=6.0, npix_side=96, nrays=60.0)
    g = mm.mm_geometry_of(mm.params(**cfg))
    rect = (37, min(g["nx"], 37 + 1000), 11, min(g["ny"], 11 + 700))      # blocks from (37, 11)
    far = dict(order=12, ratio=0.4, block_tiles=2)
    ii, jj = sample_rays(g["nx"], g["ny"], 8000, 2, rect)
    check_rays(ctx, lh, f, cfg, far, ii, jj, rect=rect)
    m = mm.mm_shoot(ctx, lh, P(cfg, far, ray_rect=rect))
    got, st = mm.mm_map_fetch(ctx, m)
    mm.mm_release_map(ctx, m)
    ref, tot, _ = oracle.far_map(ocfg(cfg), f, far, rect=rect)
    assert st["rays_shot"] == tot["shot"] == (rect[1] - rect[0]) * (rect[3] - rect[2])
    assert int(np.abs(got.astype(np.int64) - ref).sum()) <= 2 * MISBIN * tot["shot"] + 2
    mm.mm_release_lenses(ctx, lh)


@pytest.mark.parametrize("cfg,seed,n", [(CFG1, 2, 6000), (CFG2, 3, 3000)], ids=["fig1", "config2"])
def test_full_size_sampled_rays(ctx, cfg, seed, n):
    """Full-size maps: rays sampled over the whole grid, launched as mm_shoot would."""
    if cfg is CFG1:
        nstar, radius = field.nstar_rule(0.4, 0.0, 0.0, 20.0)
    else:
        nstar, radius = 25000, 250.0
    f = synth.lens_field(nstar, radius, seed)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    g = mm.mm_geometry_of(mm.params(**cfg))
    ii, jj = sample_rays(g["nx"], g["ny"], n, seed)
    err, bound = check_rays(ctx, lh, f, cfg, FAR_DEFAULT, ii, jj)
    assert bound.max() < 1e-6                                  # the default is exact to FP32 accuracy
    mm.mm_release_lenses(ctx, lh)


def test_far_map_against_the_exact_gpu_map_fig1_window(ctx):
    """The default far field reproduces the exact FP32 map: same counts but for edge rays."""
    nstar, radius = field.nstar_rule(0.4, 0.0, 0.0, 20.0)
    f = synth.lens_field(nstar, radius, 2)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    g = mm.mm_geometry_of(mm.params(**CFG1))
    c = g["nx"] // 2
    rect = (c - 4096, c + 4096, c - 4096, c + 4096)
    m_far = mm.mm_shoot(ctx, lh, P(CFG1, FAR_DEFAULT, ray_rect=rect))
    m_ex = mm.mm_shoot(ctx, lh, mm.params(**CFG1, ray_rect=rect))
    far, st_f = mm.mm_map_fetch(ctx, m_far)
    ex, st_e = mm.mm_map_fetch(ctx, m_ex)
    cmp = mm.mm_map_compare(ctx, m_far, m_ex)
    assert st_f["rays_shot"] == st_e["rays_shot"]
    assert int(np.abs(far.astype(np.int64) - ex).sum()) <= 2 * MISBIN * st_f["rays_shot"]
    assert cmp["rms_dm"] < 0.01 and cmp["ks_p"] > 0.99          # far below the shot noise 1.09 / sqrt(N)
    for m in (m_far, m_ex):
        mm.mm_release_map(ctx, m)
    mm.mm_release_lenses(ctx, lh)


def test_block_aligned_parts_equal_one_shot(ctx):
    cfg = dict(CFG0, precision=mm.MM_FAR32)
    g = mm.mm_geometry_of(mm.params(**CFG0))
    whole = mm.mm_shoot(ctx, 0, P(CFG0, FAR_DEFAULT))
    w_counts, w_st = mm.mm_map_fetch(ctx, whole)
    mm.mm_release_map(ctx, whole)
    m = mm.mm_shoot(ctx, 0, P(CFG0, FAR_DEFAULT, ray_rect=(0, 0, 0, 0)))
    bw, bh = 64 * 8, 32 * 8
    for (i0, i1) in ((0, 2 * bw), (2 * bw, g["nx"])):
        for (j0, j1) in ((0, 5 * bh), (5 * bh, g["ny"])):
            mm.mm_shoot_into(ctx, 0, P(CFG0, FAR_DEFAULT, ray_rect=(i0, i1, j0, j1)), m)
    got, st = mm.mm_map_fetch(ctx, m)
    mm.mm_release_map(ctx, m)
    assert np.array_equal(got, w_counts) and st["rays_shot"] == w_st["rays_shot"]
    assert st["far_bound"] == pytest.approx(w_st["far_bound"], rel=1e-6)
    m2 = mm.mm_map_restore(ctx, 0, P(CFG0, FAR_DEFAULT), got, st)       # a checkpoint keeps the bound
    assert mm.mm_map_fetch(ctx, m2, want_counts=False)[1]["far_bound"] == st["far_bound"]
    mm.mm_release_map(ctx, m2)
    assert cfg["precision"] == mm.MM_FAR32


def test_automatic_block_equals_the_chosen_explicit_block(ctx):
    f = field0()
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    auto = mm.params(**CFG0, precision=mm.MM_FAR32)                      # far_block = 0 by default
    m = mm.mm_shoot(ctx, lh, auto)
    got_auto, st = mm.mm_map_fetch(ctx, m)
    mm.mm_release_map(ctx, m)
    bt = st["far_block"]                                                 # chosen for these 100 lenses
    assert 1 <= bt <= 64
    m = mm.mm_shoot(ctx, lh, P(CFG0, dict(order=auto.far_order, ratio=auto.far_ratio, block_tiles=bt)))
    got, st2 = mm.mm_map_fetch(ctx, m)
    mm.mm_release_map(ctx, m)
    assert st2["far_block"] == bt
    np.testing.assert_array_equal(got_auto, got)
    # the lens field of the parameters themselves: the geometry reports the map's choice
    p = mm.params(**CFG0, precision=mm.MM_FAR32, nstar=100, disc_radius=15.81)
    m = mm.mm_shoot(ctx, 0, p)
    assert mm.mm_map_fetch(ctx, m, want_counts=False)[1]["far_block"] == mm.mm_geometry_of(p)["far_block"]
    mm.mm_release_map(ctx, m)
    mm.mm_release_lenses(ctx, lh)


def test_far_parameters_validated(ctx):
    for bad in (dict(far_order=0), dict(far_order=33), dict(far_ratio=0.0), dict(far_ratio=0.95),
                dict(far_block=-1), dict(far_block=65)):
        p = P(CFG0, FAR_DEFAULT)
        for k, v in bad.items():
            setattr(p, k, v)
        with pytest.raises(mm.MMError) as e:
            mm.mm_shoot(ctx, 0, p)
        assert e.value.code == mm.MM_EINVAL
        with pytest.raises(mm.MMError) as e:
            mm.mm_submit(ctx, 0, p)
        assert e.value.code == mm.MM_EINVAL


def test_served_far_maps_identical_to_alone(ctx):
    """Far-field requests served together with exact ones (waves carry slices of each map's
    block rows) give the maps shot alone, bit for bit."""
    mm.mm_serve_config(ctx, max_active=6, wave_ms=0.5)
    cases = [(dict(CFG0), dict(order=10, ratio=0.15, block_tiles=0)),
             (dict(CFG0, sigma=0.5, gamma=0.1), dict(order=12, ratio=0.3, block_tiles=2)),
             (dict(sigma=0.55, gamma=0.2, smooth_frac=0.3, side=6.0, npix_side=96, nrays=60.0),
              dict(order=8, ratio=0.2, block_tiles=1)),
             (dict(CFG0, sigma=0.3), None)]                                # an exact map in the mix
    f = synth.lens_field(300, 12.0, 7, model=synth.MASS_LOGNORMAL)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    reqs, alone = [], []
    for cfg, far in cases * 2:
        p = P(cfg, far) if far else mm.params(**cfg)
        m = mm.mm_shoot(ctx, lh, p)
        alone.append(mm.mm_map_fetch(ctx, m)[0].copy())
        mm.mm_release_map(ctx, m)
        reqs.append(mm.mm_submit(ctx, lh, p))
    for r, a in zip(reqs, alone):
        m = mm.mm_wait(ctx, r, timeout_s=120)
        got, st = mm.mm_map_fetch(ctx, m)
        np.testing.assert_array_equal(got, a)
        mm.mm_release_map(ctx, m)
    mm.mm_release_lenses(ctx, lh)


def test_batch_mixes_precisions(ctx):
    f = field0()
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    plist = [mm.params(**CFG0), P(CFG0, FAR_DEFAULT), mm.params(**CFG0, precision=mm.MM_FP64)]
    maps = mm.mm_shoot_batch(ctx, [lh] * 3, plist)
    ref, tot = oracle.shoot_map(ocfg(CFG0), f)
    for m in maps:
        got, st = mm.mm_map_fetch(ctx, m)
        assert st["rays_shot"] == tot["shot"]
        assert int(np.abs(got.astype(np.int64) - ref).sum()) <= 2 * MISBIN * tot["shot"]
        mm.mm_release_map(ctx, m)
    mm.mm_release_lenses(ctx, lh)


def test_near_lists_longer_than_the_staging_buffer(ctx):
    """1500 lenses all near (ratio 1e-6): every block's near list spans three shared-memory
    chunks (512 lenses each), re-staged tile by tile; the result is the exact method's."""
    f = synth.lens_field(1500, 12.0, 11)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    cfg = dict(sigma=0.4, gamma=0.1, smooth_frac=0.0, side=3.0, npix_side=64, nrays=40.0)
    far = dict(order=4, ratio=1e-6, block_tiles=2)
    g = mm.mm_geometry_of(mm.params(**cfg))
    ii, jj = sample_rays(g["nx"], g["ny"], 6000, 4)
    check_rays(ctx, lh, f, cfg, far, ii, jj)
    a_exact, _, _ = oracle.shoot_rays(ocfg(cfg), f, ii, jj)
    a_far, _ = mm.mm_debug_deflect(ctx, lh, P(cfg, far), ii, jj)
    assert np.hypot(*(a_far - a_exact).T).max() <= ALPHA_TOL
    m = mm.mm_shoot(ctx, lh, P(cfg, far))
    got, st = mm.mm_map_fetch(ctx, m)
    mm.mm_release_map(ctx, m)
    ref, tot = oracle.shoot_map(ocfg(cfg), f)
    assert st["far_bound"] == 0.0 and st["rays_shot"] == tot["shot"]
    assert int(np.abs(got.astype(np.int64) - ref).sum()) <= 2 * MISBIN * tot["shot"]
    mm.mm_release_lenses(ctx, lh)


def test_no_lenses_gives_the_smooth_map_exactly(ctx):
    """N* = 0: only the smooth convergence and shear. The far path's lens equation is the exact
    FP32 path's, so both give the oracle's integer map (parameters without rays on pixel edges)."""
    cfg = dict(sigma=0.53, gamma=0.1, smooth_frac=1.0, side=2.0, npix_side=16, nrays=121.0)
    empty = synth.lens_field(0, 1.0, 1)
    lh = mm.mm_create_lenses_from(ctx, empty.x, empty.y, empty.m)
    maps = []
    for p in (P(cfg, FAR_DEFAULT), mm.params(**cfg)):
        m = mm.mm_shoot(ctx, lh, p)
        got, st = mm.mm_map_fetch(ctx, m)
        mm.mm_release_map(ctx, m)
        maps.append((got, st))
    ref, tot = oracle.shoot_map(ocfg(cfg), empty)
    np.testing.assert_array_equal(maps[0][0], ref)
    np.testing.assert_array_equal(maps[0][0], maps[1][0])
    assert maps[0][1]["far_bound"] == 0.0 and maps[0][1]["rays_in"] == tot["inside"]
    mm.mm_release_lenses(ctx, lh)


# ---- grouped far lenses: cells of the lens tree act through their moments (Sect. 2.1) ----
# 20 000 lognormal lenses in a disc of 238 Einstein radii around a 10 x 10 R_E ray grid, blocks
# of 2 x 2 tiles: most cells are far from every block and are grouped.
CFG_G = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=4.0, npix_side=64, nrays=16.0)
FAR_GROUP = [dict(order=10, ratio=0.3, block_tiles=2, group_order=16, group_theta=0.5, group_leaf=16),
             dict(order=6, ratio=0.15, block_tiles=4, group_order=8, group_theta=0.6, group_leaf=5),
             dict(order=16, ratio=0.2, block_tiles=1, group_order=32, group_theta=0.3, group_leaf=64)]


def field_g():
    mmean = field.mean_mass(1, 0.0, 0.5)
    return synth.lens_field(20000, field.radius_for_nstar(20000, 0.4, mmean), 23, synth.MASS_LOGNORMAL)


@pytest.mark.parametrize("far", FAR_GROUP, ids=["K16", "K8-leaf5", "K32-P16"])
def test_grouped_rays_and_map_match_the_oracle(ctx, far):
    """The lens tree built on the device, the cells grouped by each block and their series agree
    with the oracle's statement of the grouped far field: per-ray deflections within 1e-5 R_E,
    pixels within the FP32 margin, the map within 2e-4 of the rays, and the bound the oracle's."""
    f = field_g()
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    g = mm.mm_geometry_of(mm.params(**CFG_G))
    ii, jj = sample_rays(g["nx"], g["ny"], 4000, 3)
    check_rays(ctx, lh, f, CFG_G, far, ii, jj)
    m = mm.mm_shoot(ctx, lh, P(CFG_G, far))
    got, st = mm.mm_map_fetch(ctx, m)
    mm.mm_release_map(ctx, m)
    ref, tot, bmax = oracle.far_map(ocfg(CFG_G), f, far)
    assert st["far_group"] == far["group_order"]
    assert st["rays_shot"] == tot["shot"] and st["rays_in"] + st["rays_out"] == st["rays_shot"]
    assert int(np.abs(got.astype(np.int64) - ref).sum()) <= 2 * MISBIN * tot["shot"]
    assert st["far_bound"] == pytest.approx(bmax, rel=2e-3)
    mm.mm_release_lenses(ctx, lh)


def test_grouped_maps_are_deterministic_and_close_to_ungrouped(ctx):
    """Grouping changes a map only within its bound: against the same map without grouping, and
    the tree walk and the moments have a fixed order, so repeated maps are identical."""
    f = field_g()
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    far = FAR_GROUP[0]
    maps = []
    for _ in range(3):
        m = mm.mm_shoot(ctx, lh, P(CFG_G, far))
        maps.append(mm.mm_map_fetch(ctx, m)[0].copy())
        mm.mm_release_map(ctx, m)
    assert np.array_equal(maps[0], maps[1]) and np.array_equal(maps[0], maps[2])
    m = mm.mm_shoot(ctx, lh, P(CFG_G, dict(far, group_order=0)))
    plain, st = mm.mm_map_fetch(ctx, m)
    mm.mm_release_map(ctx, m)
    assert int(np.abs(maps[0].astype(np.int64) - plain).sum()) <= 2 * MISBIN * st["rays_shot"]
    mm.mm_release_lenses(ctx, lh)


def test_automatic_grouping_follows_the_cost_model(ctx):
    """far_group_order = -1 and far_block = 0 (the defaults): the map takes the plan that
    mm_geometry_of reports for its lens count and disc -- here no grouping at 1e5 lenses and
    K = 24 from 1e6 on -- and the grouped rays match the oracle's statement of that plan
    (theta = 0.3, leaves of 64 lenses)."""
    cfg = dict(CFG_G, nrays=4.0)
    for n, k_expected in ((10 ** 5, 0), (10 ** 6, 24)):
        r = field.radius_for_nstar(n, 0.4)
        f = synth.lens_field(n, r, 29)
        lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
        plan = mm.mm_geometry_of(mm.params(**cfg, precision=mm.MM_FAR32, nstar=n, disc_radius=r))
        assert plan["far_group"] == k_expected
        m = mm.mm_shoot(ctx, lh, mm.params(**cfg, precision=mm.MM_FAR32))
        _, st = mm.mm_map_fetch(ctx, m, want_counts=False)
        mm.mm_release_map(ctx, m)
        assert (st["far_group"], st["far_block"]) == (plan["far_group"], plan["far_block"])
        if k_expected:
            far = dict(order=10, ratio=0.15, block_tiles=st["far_block"], group_order=24, group_theta=0.3,
                       group_leaf=64)
            g = mm.mm_geometry_of(mm.params(**cfg))
            ii, jj = sample_rays(g["nx"], g["ny"], 300, 5)
            check_rays(ctx, lh, f, cfg, far, ii, jj)
        mm.mm_release_lenses(ctx, lh)


def test_grouping_parameters_validated(ctx):
    for kw in (dict(far_group_order=33), dict(far_group_order=-2), dict(far_group_order=8, far_order=17),
               dict(far_group_theta=0.0), dict(far_group_theta=0.95), dict(far_group_leaf=0)):
        with pytest.raises(mm.MMError) as e:
            mm.mm_geometry_of(mm.params(**CFG_G, precision=mm.MM_FAR32, **kw))
        assert e.value.code == mm.MM_EINVAL
