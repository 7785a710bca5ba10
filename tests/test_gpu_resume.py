"""Shooting a map in parts and resuming it from a checkpoint (mm_shoot_into,
mm_map_restore). Counts are integers, so parts that cover the ray lattice of
Sect. 2 once and start on the 64 x 32-ray tile grid give the one-shot map bit for
bit (any cut does in FP64, whose rays do not depend on their tile); a checkpoint
fetched in one context and restored in another continues to the same map."""
import random

import numpy as np
import pytest

import oracle
import paper_1005_5198_gb300 as mm
import synth
from oracle import field

pytestmark = pytest.mark.gpu

CFG0 = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=4.0, npix_side=128, nrays=100.0)
# fewer than 2048 tiles and more than 1024 lenses: each tile's lens sum is split over CTAs
CFG_SPLIT = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=4.0, npix_side=64, nrays=100.0, nstar=3000,
                 disc_radius=8.0)
# shear and smooth matter: a 3 : 1 ray rectangle
CFG_SHEAR = dict(sigma=0.6, gamma=0.2, smooth_frac=0.3, side=8.0, npix_side=256, nrays=50.0)


@pytest.fixture(scope="module")
def ctx():
    mm.build()
    c = mm.mm_init(0)
    yield c
    mm.mm_destroy(c)


def P(cfg, **kw):
    d = dict(cfg)
    d.update(kw)
    return mm.params(**d)


def one_shot(ctx, cfg, lenses=0):
    m = mm.mm_shoot(ctx, lenses, P(cfg))
    counts, st = mm.mm_map_fetch(ctx, m)
    mm.mm_release_map(ctx, m)
    return counts, st


def parts(nx, ny, cuts_i, cuts_j, seed=0):
    """Rectangles [i0, i1, j0, j1) of the grid cut at cuts_i x cuts_j, in a shuffled order."""
    ci = [0] + list(cuts_i) + [nx]
    cj = [0] + list(cuts_j) + [ny]
    rects = [(ci[a], ci[a + 1], cj[b], cj[b + 1]) for a in range(len(ci) - 1) for b in range(len(cj) - 1)]
    random.Random(seed).shuffle(rects)
    return rects


def shoot_in_parts(ctx, cfg, rects, lenses=0):
    m = mm.mm_shoot(ctx, lenses, P(cfg, ray_rect=(0, 0, 0, 0)))     # an empty map
    for r in rects:
        mm.mm_shoot_into(ctx, 0, P(cfg, ray_rect=r), m)
    counts, st = mm.mm_map_fetch(ctx, m)
    mm.mm_release_map(ctx, m)
    return counts, st


@pytest.mark.parametrize("cfg", [CFG0, CFG_SPLIT, CFG_SHEAR], ids=["plain", "lens-split", "shear"])
def test_tile_aligned_parts_equal_one_shot(ctx, cfg):
    g = mm.mm_geometry_of(P(cfg))
    nx, ny = g["nx"], g["ny"]
    whole, st_w = one_shot(ctx, cfg)
    if cfg is CFG_SPLIT:
        assert st_w["lens_splits"] > 1
    rects = parts(nx, ny, [64 * (nx // 64 // 3), 64 * (2 * nx // 64 // 3)], [32 * (ny // 32 // 2)])
    got, st = shoot_in_parts(ctx, cfg, rects)
    assert np.array_equal(got, whole)
    for k in ("rays_shot", "rays_in", "rays_out", "interactions"):
        assert st[k] == st_w[k], k


def test_fp64_parts_at_any_cut_equal_one_shot(ctx):
    cfg = dict(CFG0, precision=mm.MM_FP64)
    g = mm.mm_geometry_of(P(cfg))
    whole, st_w = one_shot(ctx, cfg)
    got, st = shoot_in_parts(ctx, cfg, parts(g["nx"], g["ny"], [1001, 2777], [333]))
    assert np.array_equal(got, whole)
    assert st["rays_shot"] == st_w["rays_shot"] and st["rays_in"] == st_w["rays_in"]


def test_unaligned_fp32_parts_keep_oracle_parity(ctx):
    f = synth.lens_field(100, field.radius_for_nstar(100, 0.4), 1)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    g = mm.mm_geometry_of(P(CFG0))
    got, st = shoot_in_parts(ctx, CFG0, parts(g["nx"], g["ny"], [1001], [333, 2000]), lenses=lh)
    ref, tot = oracle.shoot_map(dict(CFG0, margin=1.5), f)
    assert st["rays_shot"] == tot["shot"] == g["nx"] * g["ny"]
    assert int(np.abs(got.astype(np.int64) - ref).sum()) <= 2e-4 * tot["shot"]
    mm.mm_release_lenses(ctx, lh)


def test_checkpoint_restored_in_a_new_context_resumes_bit_exact(ctx):
    cfg = CFG_SHEAR
    g = mm.mm_geometry_of(P(cfg))
    whole, st_w = one_shot(ctx, cfg)
    bands = [(0, g["nx"], j, min(j + 32 * 40, g["ny"])) for j in range(0, g["ny"], 32 * 40)]
    assert len(bands) >= 3
    done = len(bands) // 2
    a = mm.mm_init(0)
    try:
        m = mm.mm_shoot(a, 0, P(cfg, ray_rect=(0, 0, 0, 0)))
        for r in bands[:done]:
            mm.mm_shoot_into(a, 0, P(cfg, ray_rect=r), m)
        ckpt, st_ck = mm.mm_map_fetch(a, m)                  # the checkpoint: counts + stats
    finally:
        mm.mm_destroy(a)                                     # the run is interrupted
    assert st_ck["rays_shot"] == sum((r[1] - r[0]) * (r[3] - r[2]) for r in bands[:done])
    b = mm.mm_init(0)
    try:
        m = mm.mm_map_restore(b, 0, P(cfg), ckpt, st_ck)
        for r in bands[done:]:
            mm.mm_shoot_into(b, 0, P(cfg, ray_rect=r), m)
        got, st = mm.mm_map_fetch(b, m)
    finally:
        mm.mm_destroy(b)
    assert np.array_equal(got, whole)
    for k in ("rays_shot", "rays_in", "rays_out"):
        assert st[k] == st_w[k], k


def test_parts_and_checkpoints_reject_mismatches(ctx):
    m = mm.mm_shoot(ctx, 0, P(CFG0, ray_rect=(0, 64, 0, 32)))
    with pytest.raises(mm.MMError) as e:                     # another convergence
        mm.mm_shoot_into(ctx, 0, P(CFG0, sigma=0.5, ray_rect=(64, 128, 0, 32)), m)
    assert e.value.code == mm.MM_EINVAL
    with pytest.raises(mm.MMError) as e:                     # another precision
        mm.mm_shoot_into(ctx, 0, P(CFG0, precision=mm.MM_FP64, ray_rect=(64, 128, 0, 32)), m)
    assert e.value.code == mm.MM_EINVAL
    f = synth.lens_field(7, 3.0, 3)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    with pytest.raises(mm.MMError) as e:                     # a lens set of another size
        mm.mm_shoot_into(ctx, lh, P(CFG0, ray_rect=(64, 128, 0, 32)), m)
    assert e.value.code == mm.MM_EINVAL
    mm.mm_release_lenses(ctx, lh)
    counts, st = mm.mm_map_fetch(ctx, m)
    mm.mm_release_map(ctx, m)
    with pytest.raises(mm.MMError) as e:                     # a released map
        mm.mm_shoot_into(ctx, 0, P(CFG0, ray_rect=(64, 128, 0, 32)), m)
    assert e.value.code == mm.MM_ENOTFOUND
    bad = counts.copy()
    bad.flat[0] += 1                                         # counts no longer sum to rays_in
    with pytest.raises(mm.MMError) as e:
        mm.mm_map_restore(ctx, 0, P(CFG0), bad, st)
    assert e.value.code == mm.MM_EINVAL
    with pytest.raises(mm.MMError) as e:                     # another map size
        mm.mm_map_restore(ctx, 0, P(CFG0, npix_side=64), counts, st)
    assert e.value.code == mm.MM_EINVAL
    with pytest.raises(mm.MMError) as e:                     # another lattice (N_rays)
        mm.mm_map_restore(ctx, 0, P(CFG0, nrays=64.0), counts, st)
    assert e.value.code == mm.MM_EINVAL
    m2 = mm.mm_map_restore(ctx, 0, P(CFG0), counts, st)
    got, st2 = mm.mm_map_fetch(ctx, m2)
    assert np.array_equal(got, counts) and st2["rays_shot"] == st["rays_shot"] == 64 * 32
    mm.mm_release_map(ctx, m2)
