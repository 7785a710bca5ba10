"""The C-ABI library without a GPU: it loads, exports every entry point that
include/mm.h declares, validates parameters, and its host-side geometry and
lens-field rules agree with the oracle's independent implementation."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import paper_1005_5198_gb300 as mm
import synth
from oracle import field

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    mm.build()


def _declared():
    text = open(os.path.join(ROOT, "include", "mm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mm_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    names = _declared()
    assert len(names) >= 25
    lib = C.CDLL(mm.LIB)
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/mm.h but not exported"
    assert set(names) == set(mm.EXPORTED)


def test_init_without_gpu_fails_cleanly():
    with pytest.raises(mm.MMError) as e:
        mm.mm_init(0)
    assert e.value.code in (mm.MM_EDEVICE, mm.MM_EINVAL)


@pytest.mark.parametrize("bad", [
    dict(sigma=0.5, gamma=0.5), dict(sigma=0.4, gamma=0.0, side=0.0), dict(sigma=0.4, gamma=0.0, npix_side=0),
    dict(sigma=0.4, gamma=0.0, npix_side=40000), dict(sigma=0.4, gamma=0.0, nrays=0.0),
    dict(sigma=0.4, gamma=0.0, smooth_frac=1.5), dict(sigma=float("nan"), gamma=0.0),
    dict(sigma=0.4, gamma=0.0, precision=7), dict(sigma=0.4, gamma=0.0, mass_model=9),
    dict(sigma=0.4, gamma=0.0, ray_rect=(0, 10 ** 9, 0, 10)),
    dict(sigma=0.4, gamma=0.0, side=20.0, npix_side=8, nrays=1e12),
    dict(sigma=0.4, gamma=0.0, ray_mode=2),
    dict(sigma=0.4, gamma=0.0, ray_mode=1, precision=2),                      # random rays: not MM_FAR32
    dict(sigma=0.4, gamma=0.0, ray_mode=1, ray_rect=(10, 100, 0, 64)),        # random rays: tile-aligned parts
    dict(sigma=0.4, gamma=0.0, ray_mode=1, ray_rect=(64, 100, 16, 64)),
])
def test_invalid_parameters_rejected(bad):
    kw = dict(side=4.0, npix_side=64, nrays=100.0)
    kw.update(bad)
    with pytest.raises(mm.MMError) as e:
        mm.mm_geometry_of(mm.params(**kw))
    assert e.value.code == mm.MM_EINVAL


def test_random_rays_accepted_on_the_tile_grid():
    for kw in (dict(ray_mode=1), dict(ray_mode=1, precision=1), dict(ray_mode=1, ray_rect=(64, 100, 32, 64))):
        g = mm.mm_geometry_of(mm.params(sigma=0.4, gamma=0.0, side=4.0, npix_side=64, nrays=100.0, **kw))
        assert g["nx"] > 0


def test_geometry_matches_oracle_on_random_maps():
    rng = np.random.default_rng(5)
    for _ in range(300):
        s, g = rng.uniform(0, 1.6), rng.uniform(-0.7, 0.7)
        if min(abs(1 - s - g), abs(1 - s + g)) < 0.01:
            continue
        p = dict(sigma=s, gamma=g, smooth_frac=rng.uniform(0, 1), side=rng.uniform(1, 40),
                 npix_side=int(rng.integers(1, 3000)), nrays=float(rng.choice([1.0, 7.0, 100.0, 2000.0])),
                 margin=rng.uniform(1.0, 2.0))
        try:
            go = oracle.geometry(p)
        except ValueError:
            continue
        if go["nx"] > 2 ** 23 or go["ny"] > 2 ** 23 or go["width"] > 2e5 or go["height"] > 2e5:
            continue
        gp = mm.mm_geometry_of(mm.params(**p))
        for k in ("nx", "ny"):
            assert gp[k] == go[k]
        for k in ("pix", "delta", "width", "height"):
            assert gp[k] == pytest.approx(go[k], rel=1e-14)
        assert gp["mu_theory"] == pytest.approx(field.mu_theory(s, g), rel=1e-13)


def test_nstar_and_radius_rules_match_oracle():
    cases = [(0.1 * k, 0.0, 0.0) for k in range(1, 10)] + [(0.45, 0.1 * k, 0.0) for k in range(11)]
    cases += [(0.45, 0.5, 0.1 * k) for k in range(10)] + [(0.45, 0.5, 0.99)]
    for s, g, f in cases:
        for model, mmean in ((0, 1.0), (1, field.mean_mass(1, 0.0, 0.5))):
            n, r = field.nstar_rule(s, g, f, 20.0, 1.5, mmean)
            gp = mm.mm_geometry_of(mm.params(sigma=s, gamma=g, smooth_frac=f, side=20.0, npix_side=64, nrays=10.0,
                                              mass_model=model, mass_s=0.5))
            assert gp["nstar"] == n
            assert gp["disc_radius"] == pytest.approx(r, rel=1e-14)
    # N* given, R from Eq. nstar
    gp = mm.mm_geometry_of(mm.params(sigma=0.8, smooth_frac=0.5, gamma=0.3, side=40.0, npix_side=64, nrays=10.0,
                                      nstar=25000))
    assert gp["nstar"] == 25000 and gp["disc_radius"] == pytest.approx(field.radius_for_nstar(25000, 0.4), rel=1e-14)


def test_variant_table():
    n = mm.mm_variant_count()
    assert n >= 4
    names = [mm.mm_variant_name(v) for v in range(n)]
    assert len(set(names)) == n and mm.mm_variant_name(n) == "invalid"


def test_input_generator_is_independent_of_method():
    # the shared generator module draws numbers only: it must not import the oracle or the library
    src = open(os.path.join(ROOT, "synth", "__init__.py")).read()
    assert "oracle" not in re.sub(r'""".*?"""', "", src, flags=re.S)
    assert "paper_1005_5198_gb300" not in src
    f = synth.lens_field(10, 3.0, 1)
    assert f.n == 10


def test_sweep_plans_reproduce_printed_lens_counts():
    """The sweep driver's sigma and gamma sweeps use the paper's parameter grids (Sect. 3.1)."""
    from paper_1005_5198_gb300 import sweep
    printed_sigma = [65, 163, 313, 558, 987, 1817, 3701, 9343, 41257]
    got = [p["nstar"] for p in sweep.plan("sigma", 1024, 1000.0)]
    assert got[:8] == printed_sigma[:8] and abs(got[8] - printed_sigma[8]) <= 10
    printed_gamma = [741, 814, 1093, 1875, 4796, 41134, 41119, 4748, 1787, 956, 606]
    assert [p["nstar"] for p in sweep.plan("gamma", 2048, 1000.0)] == printed_gamma
    sm = sweep.plan("smooth", 2048, 1000.0)
    assert len(sm) == 11 and sm[-1]["smooth_frac"] == 0.99
    assert all(a["nstar"] >= b["nstar"] for a, b in zip(sm, sm[1:]))      # N* falls as s grows


def test_checked_build_exports_the_same_symbols():
    """The checked variant (-DMM_CHECKS) compiles and exports the ABI of the normal build."""
    import ctypes
    from paper_1005_5198_gb300 import buildlib
    path = buildlib.build(checked=True)
    lib = ctypes.CDLL(path)
    for name in mm.EXPORTED:
        assert hasattr(lib, name), name


def test_far_block_choice():
    """far_block = 0: the block side that minimises the modelled time; given sides pass through."""
    fig1 = dict(sigma=0.4, gamma=0.0, side=20.0, npix_side=1024, nrays=2000.0, precision=mm.MM_FAR32)
    assert mm.mm_geometry_of(mm.params(**fig1))["far_block"] == 8
    cfg2 = dict(sigma=0.8, gamma=0.3, smooth_frac=0.5, side=40.0, npix_side=2048, nrays=500.0, nstar=25000,
                disc_radius=250.0, precision=mm.MM_FAR32)
    assert mm.mm_geometry_of(mm.params(**cfg2))["far_block"] == 16
    counts = (10 ** 3, 10 ** 5, 10 ** 7, 10 ** 9)
    # every far lens alone: block preparation grows as blocks x N*, so more lenses want larger blocks
    alone = [mm.mm_geometry_of(mm.params(**dict(fig1, nstar=n, far_group_order=0)))["far_block"] for n in counts]
    assert alone == sorted(alone) and alone[-1] == 64
    # grouped far lenses (the default from 32768 lenses): preparation grows only with the tree's
    # depth, so the side stops growing
    grouped = [mm.mm_geometry_of(mm.params(**dict(fig1, nstar=n)))["far_block"] for n in counts]
    assert grouped == sorted(grouped) and grouped[-1] < alone[-1]
    assert mm.mm_geometry_of(mm.params(**dict(fig1, far_block=3)))["far_block"] == 3
    bad = mm.params(**fig1)
    bad.far_block = -1
    with pytest.raises(mm.MMError):
        mm.mm_geometry_of(bad)
