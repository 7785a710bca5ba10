"""The map statistics (Sect. 3.1), the extended-source convolutions and the light curves (Sect. 1) at
the size the bench times them: two 8192^2 maps at N_rays = 10, each call in its bench launch
configuration (the launch shapes depend only on N_side, the profile and its size). The maps are
seeded synthetic counts with the marginal distribution of a magnification map at that N_rays
(Poisson counts of a lognormal magnification, the second map noisier), put on the device by
mm_map_restore. The oracle takes its statistics over the whole maps, its convolutions at sampled
pixels (convolve_at), and each light-curve sample from the four pixels it needs."""
import numpy as np
import pytest

import paper_1005_5198_gb300 as mm
from oracle import extended as oext
from oracle import stats as ostats

pytestmark = pytest.mark.gpu

N, NRAYS, SIDE = 8192, 10.0, 20.0          # pixel 20 / 8192 R_E, as the bench's downstream maps
SIZE = 0.02                                # Gaussian sigma and disc radius (R_E): 67 taps per pass, radius 8 px
TRACK = ((-8.0, -3.0), (8.0, 3.0))


def restore(ctx, counts):
    """A lens-free map of the given counts (mm_map_restore); its ray grid holds their sum."""
    p = mm.params(sigma=0.9, gamma=0.05, smooth_frac=1.0, side=SIDE, npix_side=N, nrays=NRAYS)
    g = mm.mm_geometry_of(p)
    tot = int(counts.sum(dtype=np.int64))
    assert tot <= g["nx"] * g["ny"]
    st = dict(rays_shot=tot, rays_in=tot, rays_out=0, interactions=0, nx=g["nx"], ny=g["ny"], nstar=0, seconds=0.0,
              mu_mean=0.0, lens_splits=1, far_bound=0.0, far_block=0)
    return mm.mm_map_restore(ctx, 0, p, counts, st)


@pytest.fixture(scope="module")
def maps():
    mm.build()
    c = mm.mm_init(0)
    rng = np.random.default_rng(8192)
    mu = rng.lognormal(0.0, 0.6, (N, N))
    ca = rng.poisson(mu * NRAYS).astype(np.uint32)
    mu *= rng.lognormal(0.0, 0.05, mu.shape)
    cb = rng.poisson(mu * NRAYS).astype(np.uint32)
    del mu
    a, b = restore(c, ca), restore(c, cb)
    yield c, a, b, ca, cb
    mm.mm_destroy(c)


def test_compare_at_bench_size_matches_oracle(maps):
    ctx, a, b, ca, cb = maps
    got = mm.mm_map_compare(ctx, a, b)
    ref = ostats.compare(ca, NRAYS, cb, NRAYS)
    print(got, ref)
    assert ref["zero_a"] > 0 and ref["zero_b"] > 0            # empty pixels at N_rays = 10
    assert got["n_rms"] == ref["n_rms"] and got["zero_a"] == ref["zero_a"] and got["zero_b"] == ref["zero_b"]
    assert got["ks_d"] == pytest.approx(ref["ks_d"], abs=1e-15)
    assert got["ks_p"] == pytest.approx(ref["ks_p"], abs=1e-6)
    assert got["rms_dm"] == pytest.approx(ref["rms_dm"], rel=1e-9)
    assert got["mean_mu_a"] == pytest.approx(ref["mean_mu_a"], rel=1e-12)
    assert got["mean_mu_b"] == pytest.approx(ref["mean_mu_b"], rel=1e-12)


@pytest.mark.parametrize("profile", [mm.MM_PROFILE_GAUSSIAN, mm.MM_PROFILE_DISC])
def test_convolution_at_bench_size_on_sampled_pixels(maps, profile):
    """600 seeded pixels over the whole map, plus the first and last pixels with a value on a row and
    a column and their outer neighbours (NaN), against the oracle."""
    ctx, a, _, ca, _ = maps
    got = mm.mm_map_convolve(ctx, a, profile, SIZE)
    h = 33 if profile == mm.MM_PROFILE_GAUSSIAN else 8
    rng = np.random.default_rng(600 + profile)
    ii = list(rng.integers(0, N, 600)) + [h - 1, h, N - h - 1, N - h, 4000, 4000, 4000, 4000]
    jj = list(rng.integers(0, N, 600)) + [4000, 4000, 4000, 4000, h - 1, h, N - h - 1, N - h]
    ref = oext.convolve_at(ca, NRAYS, profile, SIZE, SIDE / N, ii, jj)
    g = got[np.asarray(jj), np.asarray(ii)].astype(np.float64)
    np.testing.assert_array_equal(np.isnan(g), np.isnan(ref))
    assert list(np.isnan(ref[-8:])) == [True, False, False, True] * 2
    ok = ~np.isnan(ref)
    assert ok.sum() > 550
    np.testing.assert_allclose(g[ok], ref[ok], rtol=2e-5, atol=1e-6)


@pytest.mark.parametrize("profile", [mm.MM_PROFILE_GAUSSIAN, mm.MM_PROFILE_DISC])
def test_lightcurve_at_bench_size_matches_oracle(maps, profile):
    """The bench's light curve (1000 samples across the map), which convolves only the four pixels
    around each sample, against the oracle's samples of the convolved map."""
    ctx, a, _, ca, _ = maps
    got = mm.mm_map_lightcurve(ctx, a, profile, SIZE, *TRACK, 1000)
    assert mm.mm_last_kernel_ms(ctx)[1] == 1               # the four-pixel route
    ref = oext.lightcurve_of_counts(ca, NRAYS, profile, SIZE, SIDE, *TRACK, 1000)
    assert np.isfinite(ref).all()
    np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
    np.testing.assert_allclose(got, ref, rtol=2e-5, atol=1e-6)
