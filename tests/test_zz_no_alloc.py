"""mm_shoot_noalloc: shooting for callers that cannot allocate device memory.

Such callers (code under another runtime that owns the GPU's memory, or loops
that cannot afford cudaMalloc's synchronisation) hand the library their own
device buffers; the kernel's scratch lives in a fixed array inside the library.
This file is collected last so that a run stopping at the first failure has
run every other test first. Device buffers here come from torch, as a caller
of this entry point would bring its own; the library itself allocates nothing
on this path.

Checks: on maps that mm_shoot does not split over lens segments, the counts
equal mm_shoot's on a fresh context bit for bit, on two calls in a row (the
second call must not see the first call's scratch); each map also matches the
FP64 oracle within the FP32 path's tolerance (sum |N - N_oracle| <= 2e-4 of the
rays shot); a unit-mass call without a mass array and a lens-free call (the
smooth-only map, whose count per pixel is fixed exactly by the lattice) cover
the entry point's remaining documented paths.
"""
import numpy as np
import pytest

import oracle
import paper_1005_5198_gb300 as mm
import synth

pytestmark = pytest.mark.gpu

CFG1 = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=20.0, npix_side=1024, nrays=2000.0)
MISBIN_TOL = 1e-4          # the tolerance of the other parity tests: a misbinned ray moves two counts


def _noalloc_map(torch, f, params, nside, with_masses=True):
    dev = torch.device("cuda:0")
    ptr = {}
    keep = []
    for k in ("x", "y", "m"):
        a = getattr(f, k) if f is not None else np.zeros(0)
        if k == "m" and not with_masses or a.size == 0:
            ptr[k] = 0
            continue
        t = torch.from_numpy(a).to(dev)
        keep.append(t)
        ptr[k] = t.data_ptr()
    counts = torch.full((nside * nside,), -1, dtype=torch.int32, device=dev)   # garbage to be cleared
    totals = torch.full((2,), -1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    mm.mm_shoot_noalloc(ptr["x"], ptr["y"], ptr["m"], 0 if f is None else f.n, params, counts.data_ptr(),
                        totals.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return counts.cpu().numpy().view(np.uint32).reshape(nside, nside), totals.cpu().numpy().astype(np.uint64)


def _reference_map(f, params):
    ctx = mm.mm_init(0)
    try:
        lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
        h = mm.mm_shoot(ctx, lh, params)
        counts, st = mm.mm_map_fetch(ctx, h)
        return counts.copy(), st
    finally:
        mm.mm_destroy(ctx)


def _oracle_cfg(p):
    return dict(sigma=p.sigma, gamma=p.gamma, smooth_frac=p.smooth_frac, side=p.side_re, npix_side=p.npix_side,
                nrays=p.nrays_per_pix, margin=1.5)


def _fig1_field():
    g = mm.mm_geometry_of(mm.params(**CFG1))
    return synth.lens_field(g["nstar"], g["disc_radius"], 2), g


def test_noalloc_matches_mm_shoot_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    mm.build()
    torch.cuda.init()
    f1, g = _fig1_field()
    c = g["nx"] // 2
    cases = [
        # a window of the Fig. 1 map, unit masses
        (f1, mm.params(**CFG1, ray_rect=(c - 700, c + 733, c - 500, c + 470))),
        # then a different map with lognormal masses and fewer lenses: the scratch of the
        # first call must not leak into the second
        (synth.lens_field(300, 9.0, 5, synth.MASS_LOGNORMAL),
         mm.params(sigma=0.5, gamma=0.2, smooth_frac=0.3, side=6.0, npix_side=256, nrays=50.0,
                   mass_model=mm.MM_MASS_LOGNORMAL, ray_rect=(100, 1500, 200, 1000))),
    ]
    for f, p in cases:
        nside = p.npix_side
        got, totals = _noalloc_map(torch, f, p, nside)
        ref, st = _reference_map(f, p)
        assert st["lens_splits"] == 1           # mm_shoot does not split these maps either
        np.testing.assert_array_equal(got, ref)
        assert (int(totals[0]), int(totals[1])) == (st["rays_in"], st["rays_out"])
        assert int(totals[0]) + int(totals[1]) == st["rays_shot"]
        # and the FP64 oracle on the same window
        orc, tot = oracle.shoot_map(_oracle_cfg(p), f, rect=tuple(p.ray_rect))
        assert tot["shot"] == st["rays_shot"]
        l1 = int(np.abs(got.astype(np.int64) - orc.astype(np.int64)).sum())
        assert l1 <= 2 * max(2, MISBIN_TOL * tot["shot"]), l1


def test_noalloc_unit_masses_without_a_mass_array():
    """Unit masses: the mass pointer may be NULL; the map equals the one shot with a mass array of ones."""
    torch = pytest.importorskip("torch")
    mm.build()
    f, g = _fig1_field()
    c = g["nx"] // 2
    p = mm.params(**CFG1, ray_rect=(c - 640, c + 577, c - 320, c + 351))
    got, totals = _noalloc_map(torch, f, p, p.npix_side, with_masses=False)
    ref, st = _reference_map(f, p)
    np.testing.assert_array_equal(got, ref)
    assert (int(totals[0]), int(totals[1])) == (st["rays_in"], st["rays_out"])


def test_noalloc_without_lenses_gives_the_smooth_only_map():
    """N* = 0 (null lens pointers): only the smooth matter and shear act, y = diag(a, b) x with
    a = b = 1 - sigma = 0.5. A pixel of side p maps back to a 2p square, which holds exactly
    (2 sqrt(N_rays))^2 = 400 lattice points at N_rays = 100, none of them on an edge (the
    lattice is offset by half a spacing), so every pixel counts 400 rays: mu = 1/|(1-sigma)^2 -
    gamma^2| = 4 exactly (Eq. mutheory). The shot rectangle is 1.5 L / 0.5 = 1920 spacings a side."""
    torch = pytest.importorskip("torch")
    mm.build()
    p = mm.params(sigma=0.5, gamma=0.0, smooth_frac=1.0, side=4.0, npix_side=64, nrays=100.0)
    g = mm.mm_geometry_of(p)
    assert (g["nx"], g["ny"]) == (1920, 1920)
    got, totals = _noalloc_map(torch, None, p, 64)
    assert np.all(got == 400)
    assert int(totals[0]) == 64 * 64 * 400
    assert int(totals[0]) + int(totals[1]) == 1920 * 1920


def test_noalloc_rejects_more_lenses_than_its_scratch_holds():
    torch = pytest.importorskip("torch")
    mm.build()
    dev = torch.device("cuda:0")
    buf = torch.zeros(4, dtype=torch.float64, device=dev)
    out = torch.zeros(64 * 64, dtype=torch.int32, device=dev)
    tot = torch.zeros(2, dtype=torch.int64, device=dev)
    p = mm.params(sigma=0.4, gamma=0.0, side=4.0, npix_side=64, nrays=4.0)
    with pytest.raises(mm.MMError) as e:
        mm.mm_shoot_noalloc(buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), 131073, p, out.data_ptr(),
                            tot.data_ptr(), 0)
    assert e.value.code == mm.MM_EINVAL and "131072" in str(e.value)
