"""Extended-source maps and light curves on the device (Sect. 1) against the oracle. The maps they
start from are the oracle's own maps of seeded lens fields (or seeded synthetic counts), put on the
device by mm_map_restore, so the device and the oracle convolve the same counts and none of the
oracle's input comes from the device."""
import numpy as np
import pytest

import oracle
import paper_1005_5198_gb300 as mm
import synth
from oracle import extended as oext
from oracle import field

pytestmark = pytest.mark.gpu

CFG = dict(sigma=0.45, gamma=0.2, smooth_frac=0.3, side=6.0, npix_side=256, nrays=64.0)


def oracle_map_on_device(ctx, cfg, seed):
    """The oracle's map (FP64, Sect. 2) of a seeded lens field drawn by the rules of Sect. 2 for cfg,
    put on the device by mm_map_restore. Returns the device map and the oracle's counts."""
    n, r = field.nstar_rule(cfg["sigma"], cfg["gamma"], cfg["smooth_frac"], cfg["side"])
    f = synth.lens_field(n, r, seed)
    counts, tot = oracle.shoot_map(dict(cfg, margin=1.5), f)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    p = mm.params(**cfg)
    g = mm.mm_geometry_of(p)
    st = dict(rays_shot=tot["shot"], rays_in=tot["inside"], rays_out=tot["out"], interactions=0, nx=g["nx"],
              ny=g["ny"], nstar=n, seconds=0.0, mu_mean=0.0, lens_splits=1, far_bound=0.0, far_block=0)
    return mm.mm_map_restore(ctx, lh, p, counts, st), counts


@pytest.fixture(scope="module")
def shot():
    mm.build()
    c = mm.mm_init(0)
    m, counts = oracle_map_on_device(c, CFG, 41)
    yield c, m, counts
    mm.mm_destroy(c)


@pytest.mark.parametrize("profile,size", [(mm.MM_PROFILE_GAUSSIAN, 0.05), (mm.MM_PROFILE_GAUSSIAN, 0.011),
                                          (mm.MM_PROFILE_DISC, 0.12), (mm.MM_PROFILE_DISC, 0.02)])
def test_convolved_map_matches_oracle(shot, profile, size):
    ctx, m, counts = shot
    got = mm.mm_map_convolve(ctx, m, profile, size)
    ref = oext.convolve(counts, CFG["nrays"], profile, size, CFG["side"] / CFG["npix_side"])
    np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert ok.sum() > 0.5 * ref.size
    np.testing.assert_allclose(got[ok], ref[ok], rtol=2e-5, atol=1e-6)


@pytest.mark.parametrize("nside", [203, 130])
def test_convolution_of_sides_not_multiple_of_4(nside):
    """Sides that are not multiples of 4 (the tiled Gaussian then copies 4-byte words instead of
    16-byte groups and stores its outputs one by one) and leave ragged tiles: against the oracle."""
    mm.build()
    c = mm.mm_init(0)
    try:
        cfg = dict(CFG, npix_side=nside, side=6.0 * nside / 256)
        m, counts = oracle_map_on_device(c, cfg, 47)
        for profile, size in ((mm.MM_PROFILE_GAUSSIAN, 0.05), (mm.MM_PROFILE_DISC, 0.12)):
            got = mm.mm_map_convolve(c, m, profile, size)
            ref = oext.convolve(counts, cfg["nrays"], profile, size, cfg["side"] / nside)
            np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
            ok = ~np.isnan(ref)
            assert ok.sum() > 0.5 * ref.size
            np.testing.assert_allclose(got[ok], ref[ok], rtol=2e-5, atol=1e-6)
    finally:
        mm.mm_destroy(c)


def test_lightcurve_matches_oracle(shot):
    ctx, m, counts = shot
    start, end = (-2.5, -1.7), (2.3, 2.6)           # runs off the valid region at both ends
    got = mm.mm_map_lightcurve(ctx, m, mm.MM_PROFILE_GAUSSIAN, 0.04, start, end, 500)
    field_ref = oext.convolve(counts, CFG["nrays"], 0, 0.04, CFG["side"] / CFG["npix_side"])
    ref = oext.lightcurve(field_ref, CFG["side"], start, end, 500)
    np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert ok.sum() > 300
    np.testing.assert_allclose(got[ok], ref[ok], rtol=2e-5, atol=1e-6)


def test_disc_wait_that_runs_out_reports_a_device_error(shot):
    """The tiled disc kernel stages the tiles that lie inside the map by bulk copies and waits for them on
    an mbarrier with a time limit. With those copies withheld (test hook), the waits give up after their
    limit (about a second), the call returns MM_EDEVICE instead of hanging, and the same context then
    convolves correctly. The 256^2 map at radius 5 pixels has four such tiles."""
    ctx, m, counts = shot
    mm.mm_debug_inject(ctx, mm.MM_INJECT_DISC_NO_COPY)
    mm.mm_map_convolve(ctx, m, mm.MM_PROFILE_GAUSSIAN, 0.05)    # another kind of call leaves it armed
    with pytest.raises(mm.MMError) as e:
        mm.mm_map_convolve(ctx, m, mm.MM_PROFILE_DISC, 0.12)
    assert e.value.code == mm.MM_EDEVICE
    got = mm.mm_map_convolve(ctx, m, mm.MM_PROFILE_DISC, 0.12)  # the hook is one-shot
    ref = oext.convolve(counts, CFG["nrays"], mm.MM_PROFILE_DISC, 0.12, CFG["side"] / CFG["npix_side"])
    np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    np.testing.assert_allclose(got[ok], ref[ok], rtol=2e-5, atol=1e-6)


def test_profile_wider_than_map_rejected(shot):
    ctx, m, _ = shot
    with pytest.raises(mm.MMError) as e:
        mm.mm_map_convolve(ctx, m, mm.MM_PROFILE_DISC, 10.0)
    assert e.value.code == mm.MM_EINVAL


# Wide supports: the tiled kernels stage their tiles in shared memory, two tiles of a Gaussian pass
# in at most 200 KB (up to a half-width of 131 pixels) and a disc's tile with its staging buffer in
# 72 KB (up to a radius of 15 pixels); wider supports run the untiled kernels. Sizes on both sides of
# each limit, on a 320^2 map.
CFG_WIDE = dict(CFG, npix_side=320, side=7.5)            # pixel 0.0234375 R_E


@pytest.fixture(scope="module")
def shot_wide():
    mm.build()
    c = mm.mm_init(0)
    m, counts = oracle_map_on_device(c, CFG_WIDE, 43)
    yield c, m, counts
    mm.mm_destroy(c)


@pytest.mark.parametrize("profile,size,half_width", [
    (mm.MM_PROFILE_GAUSSIAN, 0.7177734375, 123), (mm.MM_PROFILE_GAUSSIAN, 0.7646484375, 131),
    (mm.MM_PROFILE_GAUSSIAN, 0.7705078125, 132),
    (mm.MM_PROFILE_DISC, 0.3633, 15), (mm.MM_PROFILE_DISC, 0.5039, 21)])
def test_wide_supports_match_oracle(shot_wide, profile, size, half_width):
    ctx, m, counts = shot_wide
    pix = CFG_WIDE["side"] / CFG_WIDE["npix_side"]
    h = int(np.ceil(4.0 * size / pix)) if profile == mm.MM_PROFILE_GAUSSIAN else int(np.floor(size / pix))
    assert h == half_width
    got = mm.mm_map_convolve(ctx, m, profile, size)
    ref = oext.convolve(counts, CFG_WIDE["nrays"], profile, size, pix)
    np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert ok.sum() == (CFG_WIDE["npix_side"] - 2 * h) ** 2
    np.testing.assert_allclose(got[ok], ref[ok], rtol=2e-5, atol=1e-6)


def test_disc_tiles_with_large_counts_use_64_bit_sums():
    """The tiled disc kernel takes each tile's row prefix sums in 32 bits and adds an output's spans
    in 32 bits while every count of the tile is below 2^32 / (2H + 1)^2, in 64 bits while below
    2^32 / (2H + 1), and otherwise stages the tile again as 64-bit prefix sums. A seeded synthetic
    map (put on the device by mm_map_restore) with a few pixels above each bound, convolved with a
    disc of radius 8 pixels (under the tiled limit of 15), has tiles of all three kinds in one
    launch; all match the oracle."""
    mm.build()
    c = mm.mm_init(0)
    try:
        n, nrays, side = 256, 1.0e6, 4.0
        pix = side / n
        size = 8.5 * pix                                   # H = 8: bound 2^32 / 17 = 252645135
        rng = np.random.default_rng(5)
        counts = rng.poisson(1000.0, (n, n)).astype(np.uint32)
        counts[10:14, 20:22] = np.uint32(300_000_000)      # 8 pixels above the bound: 64-bit prefix sums
        counts[200:202, 150:152] = np.uint32(50_000_000)   # above 2^32 / 17^2: 32-bit spans added in 64 bits
        p = mm.params(sigma=0.4, gamma=0.0, smooth_frac=1.0, side=side, npix_side=n, nrays=nrays)
        g = mm.mm_geometry_of(p)
        tot = int(counts.sum(dtype=np.int64))
        assert tot <= g["nx"] * g["ny"]
        st = dict(rays_shot=tot, rays_in=tot, rays_out=0, interactions=0, nx=g["nx"], ny=g["ny"], nstar=0,
                  seconds=0.0, mu_mean=0.0, lens_splits=1, far_bound=0.0, far_block=0)
        m = mm.mm_map_restore(c, 0, p, counts, st)
        got = mm.mm_map_convolve(c, m, mm.MM_PROFILE_DISC, size)
        ref = oext.convolve(counts, nrays, mm.MM_PROFILE_DISC, size, pix)
        np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
        ok = ~np.isnan(ref)
        assert ok.sum() == (n - 16) ** 2
        np.testing.assert_allclose(got[ok], ref[ok], rtol=2e-6, atol=1e-9)
        assert np.nanmax(ref) > 100 * np.nanmedian(ref)     # the large pixels reach some outputs
    finally:
        mm.mm_destroy(c)


# Light curves: a sample needs the convolved map at four pixels only, and when that is less work the
# library convolves just those (one CTA per sample) instead of the whole map. Both routes must give
# the pixels of mm_map_convolve bit for bit.

def _centre_track(n, side, i0, j, steps):
    """A track along pixel row j from the centre of pixel i0 to that of pixel i0 + steps. With a pixel
    and a step count that are exact binary fractions, every sample lies exactly on a pixel centre, so
    the bilinear weights are 0 and each sample is the convolved pixel itself."""
    p = side / n
    y = lambda i: -side / 2 + (i + 0.5) * p
    return (y(i0), y(j)), (y(i0 + steps), y(j))


@pytest.mark.parametrize("profile,size", [(mm.MM_PROFILE_GAUSSIAN, 0.05), (mm.MM_PROFILE_DISC, 0.12)])
def test_lightcurve_on_pixel_centres_equals_the_convolved_map(shot, profile, size):
    ctx, m, _ = shot
    conv = mm.mm_map_convolve(ctx, m, profile, size)
    i0, j, steps = 40, 100, 64
    start, end = _centre_track(CFG["npix_side"], CFG["side"], i0, j, steps)
    got = mm.mm_map_lightcurve(ctx, m, profile, size, start, end, steps + 1)
    assert mm.mm_last_kernel_ms(ctx)[1] == 1            # the four-pixel route: one kernel
    assert np.isfinite(got).all()
    np.testing.assert_array_equal(got, conv[j, i0:i0 + steps + 1].astype(np.float64))


@pytest.mark.parametrize("profile,size", [(mm.MM_PROFILE_GAUSSIAN, 0.7705078125), (mm.MM_PROFILE_DISC, 0.5039)])
def test_lightcurve_of_wide_supports_on_pixel_centres(shot_wide, profile, size):
    """Supports past the tiled kernels' limits (Gaussian half-width 132: 265 taps, more than one round
    of the four-pixel kernel's column sums; disc radius 21 pixels)."""
    ctx, m, _ = shot_wide
    conv = mm.mm_map_convolve(ctx, m, profile, size)
    i0, j, steps = 140, 160, 32
    start, end = _centre_track(CFG_WIDE["npix_side"], CFG_WIDE["side"], i0, j, steps)
    got = mm.mm_map_lightcurve(ctx, m, profile, size, start, end, steps + 1)
    assert np.isfinite(got).all()
    np.testing.assert_array_equal(got, conv[j, i0:i0 + steps + 1].astype(np.float64))


@pytest.mark.parametrize("profile,size", [(mm.MM_PROFILE_GAUSSIAN, 0.015), (mm.MM_PROFILE_DISC, 0.08)])
def test_lightcurve_routes_agree_and_match_oracle(profile, size):
    """On a 64^2 map (Gaussian half-width 3; disc radius 3 pixels, 37 taps), 300 samples are less work
    than the whole convolution and take the four-pixel route; 599 samples are more and take the
    whole-map route. Sample 2k of the second track is sample k of the first (the same t in FP64), so
    the two routes must agree bit for bit there; both match the oracle, NaN where the support leaves
    the map."""
    mm.build()
    c = mm.mm_init(0)
    try:
        cfg = dict(CFG, npix_side=64, side=1.5)
        m, counts = oracle_map_on_device(c, cfg, 53)
        start, end = (-0.7, -0.6), (0.65, 0.7)
        few = mm.mm_map_lightcurve(c, m, profile, size, start, end, 300)
        few_launches = mm.mm_last_kernel_ms(c)[1]
        many = mm.mm_map_lightcurve(c, m, profile, size, start, end, 599)
        many_launches = mm.mm_last_kernel_ms(c)[1]
        if profile == mm.MM_PROFILE_GAUSSIAN:               # one kernel, or the two convolution passes
            assert (few_launches, many_launches) == (1, 2)
        np.testing.assert_array_equal(few, many[::2])
        pix = cfg["side"] / cfg["npix_side"]
        field_ref = oext.convolve(counts, cfg["nrays"], profile, size, pix)
        for got, npts in ((few, 300), (many, 599)):
            ref = oext.lightcurve(field_ref, cfg["side"], start, end, npts)
            np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
            ok = ~np.isnan(ref)
            assert 0.5 * npts < ok.sum() < npts
            np.testing.assert_allclose(got[ok], ref[ok], rtol=2e-5, atol=1e-6)
    finally:
        mm.mm_destroy(c)
