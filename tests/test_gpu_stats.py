"""Device map statistics (Sect. 3.1) against the oracle's, and the paper's agreement test
applied to the FP32 and FP64 paths."""
import numpy as np
import pytest

import oracle
import paper_1005_5198_gb300 as mm
import synth
from oracle import field
from oracle import stats as ostats

pytestmark = pytest.mark.gpu

CFG = dict(sigma=0.45, gamma=0.2, smooth_frac=0.3, side=6.0, npix_side=256, nrays=64.0)


@pytest.fixture(scope="module")
def ctx():
    mm.build()
    c = mm.mm_init(0)
    yield c
    mm.mm_destroy(c)


def restore_counts(ctx, counts, nrays, side=6.0):
    """A map on the device holding the given host counts (mm_map_restore of a lens-free map whose
    totals are the counts' sum): seeded synthetic input for the downstream kernels."""
    n = counts.shape[0]
    # sigma = 0.9, gamma = 0.05: a ray grid 300 N_side^2 N_rays large, room for any test's counts
    p = mm.params(sigma=0.9, gamma=0.05, smooth_frac=1.0, side=side, npix_side=n, nrays=nrays)
    g = mm.mm_geometry_of(p)
    tot = int(counts.sum(dtype=np.int64))
    assert tot <= g["nx"] * g["ny"]
    st = dict(rays_shot=tot, rays_in=tot, rays_out=0, interactions=0, nx=g["nx"], ny=g["ny"], nstar=0, seconds=0.0,
              mu_mean=0.0, lens_splits=1, far_bound=0.0, far_block=0)
    return mm.mm_map_restore(ctx, 0, p, counts, st)


# The device keeps histograms of the counts below 1024 in shared memory, sends counts below
# T = 4096 (at these N_rays) to global histograms and lists the larger ones (room for
# max(4096, N_side^2 / 64) per map), widening the histograms afterwards; when a list runs out of
# room, a second pass over the maps builds the wide histograms. Seeded synthetic count maps (put on
# the device by mm_map_restore, as restore_counts above) cover each way: only small counts; a tail
# up to about 10^5 on 2 % of the pixels (listed); the same tail on 12 % of a 256^2 map (about 7900
# pixels above T, more than the list holds). All have empty pixels and different N_rays.
@pytest.mark.parametrize("nside,tail", [(256, 0.0), (192, 0.02), (256, 0.12)])
def test_compare_matches_oracle_statistics(ctx, nside, tail):
    rng = np.random.default_rng(nside + int(100 * tail))
    mu = rng.lognormal(0.0, 0.6, (nside, nside))
    if tail:
        mu[rng.random((nside, nside)) < tail] *= 300.0
    nrays_a, nrays_b = 32.0, 25.0
    ca = rng.poisson(mu * nrays_a).astype(np.uint32)
    cb = rng.poisson(mu * nrays_b * rng.lognormal(0.0, 0.05, mu.shape)).astype(np.uint32)   # a noisier map
    ca.ravel()[rng.integers(0, nside * nside, 5)] = 0                                        # empty pixels
    cb.ravel()[rng.integers(0, nside * nside, 9)] = 0
    assert (int(max(ca.max(), cb.max())) >= 4096) == (tail > 0)
    big = int(np.sum(ca >= 4096))
    assert (big > max(4096, nside * nside // 64)) == (tail > 0.1)
    assert (ca == 0).any() and (cb == 0).any()
    a = restore_counts(ctx, ca, nrays_a)
    b = restore_counts(ctx, cb, nrays_b)
    got = mm.mm_map_compare(ctx, a, b)
    ref = ostats.compare(ca, nrays_a, cb, nrays_b)
    print(got, ref)
    assert got["ks_d"] == pytest.approx(ref["ks_d"], abs=1e-15)
    assert got["n_rms"] == ref["n_rms"] and got["zero_a"] == ref["zero_a"] and got["zero_b"] == ref["zero_b"]
    assert got["rms_dm"] == pytest.approx(ref["rms_dm"], rel=1e-9)
    assert got["ks_p"] == pytest.approx(ref["ks_p"], abs=1e-6)
    assert got["mean_mu_a"] == pytest.approx(ref["mean_mu_a"], rel=1e-12)
    same = mm.mm_map_compare(ctx, a, a)
    assert same["rms_dm"] == 0.0 and same["ks_d"] == 0.0 and same["ks_p"] == pytest.approx(1.0)
    for m in (a, b):
        mm.mm_release_map(ctx, m)


def test_compare_wait_that_runs_out_reports_a_device_error(ctx):
    """The comparison streams the maps through shared memory and waits on mbarriers for the bulk copies.
    With the copies withheld (test hook), every wait gives up after its limit (about a second), the call
    returns MM_EDEVICE instead of hanging, and the same context then compares correctly."""
    rng = np.random.default_rng(5)
    ca = rng.poisson(20.0, (128, 128)).astype(np.uint32)
    cb = rng.poisson(20.0, (128, 128)).astype(np.uint32)
    a, b = restore_counts(ctx, ca, 20.0), restore_counts(ctx, cb, 20.0)
    mm.mm_debug_inject(ctx, mm.MM_INJECT_COMPARE_NO_COPY)
    with pytest.raises(mm.MMError) as e:
        mm.mm_map_compare(ctx, a, b)
    assert e.value.code == mm.MM_EDEVICE
    got = mm.mm_map_compare(ctx, a, b)                      # the hook is one-shot; the context still works
    ref = ostats.compare(ca, 20.0, cb, 20.0)
    assert got["ks_d"] == pytest.approx(ref["ks_d"], abs=1e-15)
    assert got["rms_dm"] == pytest.approx(ref["rms_dm"], rel=1e-9)
    with pytest.raises(mm.MMError):
        mm.mm_debug_inject(ctx, 99)
    for m in (a, b):
        mm.mm_release_map(ctx, m)


def test_fp32_and_fp64_maps_agree_excellently(ctx):
    """The paper's criterion for 'excellent agreement' (RMS < 0.2 mag, K-S probability > 99.7 %)
    between the compensated FP32 path and the plain FP64 path on a config-0 map."""
    cfg = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=4.0, npix_side=128, nrays=100.0)
    f = synth.lens_field(100, field.radius_for_nstar(100, 0.4), 1)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    a = mm.mm_shoot(ctx, lh, mm.params(**cfg))
    b = mm.mm_shoot(ctx, lh, mm.params(**cfg, precision=mm.MM_FP64))
    r = mm.mm_map_compare(ctx, a, b)
    print(r)
    assert r["rms_dm"] < 0.2 and r["ks_p"] > 0.997
    assert r["rms_dm"] < 1e-3           # in fact only a few rays per million differ
    for m in (a, b):
        mm.mm_release_map(ctx, m)


@pytest.mark.parametrize("nside,lam", [(129, 3.0), (256, 400.0)])
def test_normalised_map_matches_oracle(ctx, nside, lam):
    """mm_map_fetch_mu against the estimator mu = N / N_rays and Eq. deltam (oracle, FP64) on a seeded
    synthetic count map with empty pixels, a few counts above 2^24 (not exact in FP32) and an odd side
    (N_side^2 not a multiple of 4). Empty pixels are clamped to one ray for Delta m and counted.
    Bars (FP32 arithmetic): mu within 2e-7 relative (the count's and the product's roundings),
    Delta m within 1e-5 mag (log10f's 2-ulp error on values up to about 9, the subtraction and the
    final product: about 7e-6 at most)."""
    rng = np.random.default_rng(nside)
    counts = rng.poisson(lam, (nside, nside)).astype(np.uint32)
    counts.ravel()[rng.integers(0, nside * nside, 7)] = np.uint32(123_456_789)
    nrays = 1.0e4 + lam                     # ray grid large enough to hold the counts' sum
    m = restore_counts(ctx, counts, nrays)
    mu, empty = mm.mm_map_fetch_mu(ctx, m, mm.MM_MAP_MU)
    assert empty == int(np.sum(counts == 0)) and (lam > 100 or empty > 0)
    np.testing.assert_allclose(mu, counts.astype(np.float64) / nrays, rtol=2e-7, atol=0)
    dm, empty2 = mm.mm_map_fetch_mu(ctx, m, mm.MM_MAP_DELTA_M)
    assert empty2 == empty
    ref = ostats.delta_m(np.maximum(counts, 1), nrays)
    np.testing.assert_allclose(dm, ref, rtol=0, atol=1e-5)
    with pytest.raises(mm.MMError):
        mm.mm_map_fetch_mu(ctx, m, 7)
    mm.mm_release_map(ctx, m)
