"""The C ABI's tuning and error paths on the GPU: every failure is made on the host
(bad arguments, a tiny HBM budget, released handles) and reported as a status."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1005_5198_gb300 as mm
import synth
from oracle import field

pytestmark = pytest.mark.gpu

CFG0 = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=4.0, npix_side=128, nrays=100.0)


@pytest.fixture(scope="module")
def ctx():
    mm.build()
    c = mm.mm_init(0)
    yield c
    mm.mm_destroy(c)


def test_autotune_picks_a_layout_and_variant_and_keeps_parity(ctx):
    p = mm.params(sigma=0.4, gamma=0.0, side=20.0, npix_side=1024, nrays=2000.0)
    v = mm.mm_autotune(ctx, p)
    assert 0 <= v < mm.mm_variant_count()
    assert 0 <= mm.mm_get_layout(ctx) < mm.mm_layout_count()
    f = synth.lens_field(100, field.radius_for_nstar(100, 0.4), 1)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    m = mm.mm_shoot(ctx, lh, mm.params(**CFG0))
    got, st = mm.mm_map_fetch(ctx, m)
    ref, tot = oracle.shoot_map(dict(CFG0, margin=1.5), f)
    assert int(np.abs(got.astype(np.int64) - ref).sum()) <= 2e-4 * tot["shot"]
    mm.mm_release_map(ctx, m)
    mm.mm_set_layout(ctx, 1)


def test_bad_lens_arrays_rejected(ctx):
    for bad in (np.array([0.0, np.nan]), np.array([0.0, 2e5])):
        with pytest.raises(mm.MMError) as e:
            mm.mm_create_lenses_from(ctx, bad, np.zeros(2), np.ones(2))
        assert e.value.code == mm.MM_EINVAL
    with pytest.raises(mm.MMError):
        mm.mm_create_lenses_from(ctx, np.zeros(2), np.zeros(2), np.array([1.0, -1.0]))


def test_released_handles_and_buffer_sizes(ctx):
    f = synth.lens_field(10, 3.0, 2)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    m = mm.mm_shoot(ctx, lh, mm.params(**CFG0, nstar=10))
    buf = np.zeros(7, dtype=np.uint32)                      # the C call checks n_elems itself
    rc = mm.lib().mm_map_fetch(ctx.handle, m, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), 7, None)
    assert rc == mm.MM_EINVAL
    with pytest.raises(ValueError):
        mm.mm_map_fetch(ctx, m, counts=buf)
    mm.mm_release_map(ctx, m)
    with pytest.raises(mm.MMError) as e:
        mm.mm_release_map(ctx, m)
    assert e.value.code == mm.MM_ENOTFOUND
    mm.mm_release_lenses(ctx, lh)
    with pytest.raises(mm.MMError) as e:
        mm.mm_lenses_fetch(ctx, lh)
    assert e.value.code == mm.MM_ENOTFOUND


def test_ray_outside_the_grid_rejected(ctx):
    g = mm.mm_geometry_of(mm.params(**CFG0))
    with pytest.raises(mm.MMError) as e:
        mm.mm_debug_deflect(ctx, 0, mm.params(**CFG0, nstar=10), [g["nx"]], [0])
    assert e.value.code == mm.MM_EINVAL


def test_over_budget_shoot_reports_enomem():
    mm.build()
    c = mm.mm_init(0, hbm_budget_bytes=8 << 20)
    try:
        with pytest.raises(mm.MMError) as e:
            mm.mm_shoot(c, 0, mm.params(sigma=0.4, gamma=0.0, side=8.0, npix_side=4096, nrays=0.01, nstar=10))
        assert e.value.code == mm.MM_ENOMEM                   # a 64 MiB map over an 8 MiB budget
        m = mm.mm_shoot(c, 0, mm.params(**CFG0, nstar=10))   # the context stays usable
        _, st = mm.mm_map_fetch(c, m, want_counts=False)
        assert st["rays_shot"] == st["rays_in"] + st["rays_out"]
    finally:
        mm.mm_destroy(c)


def test_fp64_with_lognormal_masses_matches_oracle(ctx):
    cfg = dict(sigma=0.6, gamma=0.15, smooth_frac=0.4, side=3.0, npix_side=64, nrays=25.0)
    f = synth.lens_field(300, 8.0, 13, synth.MASS_LOGNORMAL)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    g = oracle.geometry(dict(cfg, margin=1.5))
    rect = (g["nx"] // 2 - 100, g["nx"] // 2 + 100, g["ny"] // 2 - 80, g["ny"] // 2 + 80)
    m = mm.mm_shoot(ctx, lh, mm.params(**cfg, precision=mm.MM_FP64, ray_rect=rect))
    got, st = mm.mm_map_fetch(ctx, m)
    ref, tot = oracle.shoot_map(dict(cfg, margin=1.5), f, rect=rect)
    assert int(np.abs(got.astype(np.int64) - ref).sum()) <= 2
    assert st["rays_in"] + st["rays_out"] == tot["shot"]
