"""The seeded input generator: published SplitMix64 outputs and field shape."""
import numpy as np

import synth


def test_splitmix64_published_first_outputs():
    # SplitMix64 seeded with 0: the first outputs of the reference generator of
    # Steele, Lea & Flood (2014) as distributed with its public test vectors.
    z = synth.splitmix64(0, np.arange(1, 4, dtype=np.uint64))
    assert [hex(int(v)) for v in z] == ["0xe220a8397b1dcdaf", "0x6e789e6aa1b965f4", "0x6c45d188009454f"]
    assert synth.mix64(synth.GOLDEN_GAMMA) == 0xE220A8397B1DCDAF


def test_lens_field_in_disc_uniform_and_deterministic():
    f = synth.lens_field(20000, 10.0, 3)
    g = synth.lens_field(20000, 10.0, 3)
    np.testing.assert_array_equal(f.x, g.x)
    r2 = f.x ** 2 + f.y ** 2
    assert r2.max() < 100.0
    # uniform in a disc: r^2 / R^2 is uniform on [0, 1)
    assert abs((r2 / 100.0).mean() - 0.5) < 0.01
    assert abs(f.x.mean()) < 0.1 and abs(f.y.mean()) < 0.1
    assert np.all(f.m == 1.0)
    h = synth.lens_field(20000, 10.0, 4)
    assert not np.array_equal(f.x, h.x)


def test_map_mix_guard_and_ranges():
    draws = synth.map_mix(64, 4)
    assert len(draws) == 64
    for d in draws:
        assert 0.2 <= d.sigma <= 1.5 and 0.0 <= d.gamma <= 0.6 and 0.0 <= d.smooth_frac <= 0.9
        assert min(abs(1 - d.sigma - d.gamma), abs(1 - d.sigma + d.gamma)) >= 0.05
        assert d.npix_side in (256, 512, 1024) and d.nrays in (100.0, 300.0, 1000.0)


def test_poisson_arrivals_rate():
    t = synth.poisson_arrivals(20000, 20.0, 9)
    assert np.all(np.diff(t) > 0)
    assert abs(20000 / t[-1] / 20.0 - 1.0) < 0.03
