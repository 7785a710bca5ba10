"""mm_shoot_noalloc: shooting for callers that cannot allocate device memory.

Such callers (code under another runtime that owns the GPU's memory, or loops
that cannot afford cudaMalloc's synchronisation) hand the library their own
device buffers; the kernel's scratch lives in a fixed array inside the library.
This file is collected last so that a run stopping at the first failure has
run every other test first. Device buffers here come from torch, as a caller
of this entry point would bring its own; the library itself allocates nothing
on this path.
"""
import numpy as np
import pytest

import oracle  # noqa: F401  (not used: parity here is against the existing entry point)
import paper_1005_5198_gb300 as mm
import synth
from oracle import field

pytestmark = pytest.mark.gpu

CFG1 = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=20.0, npix_side=1024, nrays=2000.0)
MISBIN_TOL = 1e-4          # the tolerance of the other parity tests: a misbinned ray moves two counts


def _noalloc_map(torch, f, params, nside):
    dev = torch.device("cuda:0")
    x = torch.from_numpy(f.x).to(dev)
    y = torch.from_numpy(f.y).to(dev)
    m = torch.from_numpy(f.m).to(dev)
    counts = torch.full((nside * nside,), -1, dtype=torch.int32, device=dev)   # garbage to be cleared
    totals = torch.full((2,), -1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    mm.mm_shoot_noalloc(x.data_ptr(), y.data_ptr(), m.data_ptr(), f.n, params, counts.data_ptr(),
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


def test_noalloc_matches_mm_shoot_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    mm.build()
    torch.cuda.init()
    n1, r1 = field.nstar_rule(0.4, 0.0, 0.0, 20.0)
    g = mm.mm_geometry_of(mm.params(**CFG1))
    c = g["nx"] // 2
    cases = [
        # a window of the Fig. 1 map, unit masses
        (synth.lens_field(n1, r1, 2), mm.params(**CFG1, ray_rect=(c - 700, c + 733, c - 500, c + 470))),
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
        shot = st["rays_shot"]
        l1 = int(np.abs(got.astype(np.int64) - ref.astype(np.int64)).sum())
        assert l1 <= 2 * MISBIN_TOL * shot, l1
        assert int(totals[0]) + int(totals[1]) == shot
        assert int(got.sum(dtype=np.int64)) == int(totals[0])
        assert abs(int(totals[0]) - st["rays_in"]) <= MISBIN_TOL * shot


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
