"""Drive every shooting path through the checked build (run as a script by
test_gpu_checked.py, in its own process: the checked library must be the first
one loaded). Any failed bounds check surfaces as MMError (MM_EDEVICE) and ends
the script with a non-zero status; results are also compared with the oracle."""
import sys

import numpy as np

import oracle
import paper_1005_5198_gb300 as mm
import synth
from oracle import field

CFG0 = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=4.0, npix_side=128, nrays=100.0)
SPLIT = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=4.0, npix_side=64, nrays=100.0)


def close(got, ref, shot, what):
    l1 = int(np.abs(got.astype(np.int64) - ref.astype(np.int64)).sum())
    assert l1 <= max(2, 4e-4 * shot), (what, l1)


def main():
    mm.use_checked_build()
    ctx = mm.mm_init(0)
    try:
        f = synth.lens_field(100, field.radius_for_nstar(100, 0.4), 1)
        lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
        ref, tot = oracle.shoot_map(dict(CFG0, margin=1.5), f)
        for prec in (mm.MM_FP32C, mm.MM_FP64, mm.MM_FAR32):             # the three kernels
            m = mm.mm_shoot(ctx, lh, mm.params(**CFG0, precision=prec))
            got, st = mm.mm_map_fetch(ctx, m)
            mm.mm_release_map(ctx, m)
            close(got, ref, tot["shot"], prec)
        # lens-split tiles, lognormal masses
        big = synth.lens_field(3000, 10.0, 5, model=synth.MASS_LOGNORMAL)
        lb = mm.mm_create_lenses_from(ctx, big.x, big.y, big.m)
        m = mm.mm_shoot(ctx, lb, mm.params(**SPLIT))
        got, st = mm.mm_map_fetch(ctx, m)
        mm.mm_release_map(ctx, m)
        assert st["lens_splits"] > 1
        ref_b, tot_b = oracle.shoot_map(dict(SPLIT, margin=1.5), big)
        close(got, ref_b, tot_b["shot"], "split")
        # far field with every lens near (near lists over several staging chunks)
        m = mm.mm_shoot(ctx, lb, mm.params(**SPLIT, precision=mm.MM_FAR32, far_ratio=1e-6, far_block=2))
        got, st = mm.mm_map_fetch(ctx, m)
        mm.mm_release_map(ctx, m)
        close(got, ref_b, tot_b["shot"], "far, all near")
        # grouped far lenses (the lens tree's walk writes the near lists under the checks)
        gf = synth.lens_field(6000, 40.0, 9, model=synth.MASS_LOGNORMAL)
        lg = mm.mm_create_lenses_from(ctx, gf.x, gf.y, gf.m)
        pg = mm.params(**SPLIT, precision=mm.MM_FAR32, far_block=2, far_group_order=12, far_group_theta=0.5,
                       far_group_leaf=8)
        m = mm.mm_shoot(ctx, lg, pg)
        got, st = mm.mm_map_fetch(ctx, m)
        mm.mm_release_map(ctx, m)
        ref_g, tot_g, _ = oracle.far_map(dict(SPLIT, margin=1.5), gf, dict(order=10, ratio=0.15, block_tiles=2,
                                                                             group_order=12, group_theta=0.5,
                                                                             group_leaf=8))
        assert st["far_group"] == 12
        close(got, ref_g, tot_g["shot"], "far, grouped")
        mm.mm_release_lenses(ctx, lg)
        # mixed batch, debug dump, parts
        maps = mm.mm_shoot_batch(ctx, [lh, lb, lh], [mm.params(**CFG0), mm.params(**SPLIT),
                                                    mm.params(**CFG0, precision=mm.MM_FAR32)])
        for h in maps:
            mm.mm_release_map(ctx, h)
        ii = np.arange(0, 3000, 7)
        for prec in (mm.MM_FP32C, mm.MM_FAR32):
            mm.mm_debug_deflect(ctx, lh, mm.params(**CFG0, precision=prec), ii, ii)
        m = mm.mm_shoot(ctx, lh, mm.params(**CFG0, ray_rect=(0, 0, 0, 0)))
        mm.mm_shoot_into(ctx, 0, mm.params(**CFG0, ray_rect=(0, 3200, 0, 1600)), m)
        mm.mm_shoot_into(ctx, 0, mm.params(**CFG0, ray_rect=(0, 3200, 1600, 3200)), m)
        got, st = mm.mm_map_fetch(ctx, m)
        mm.mm_release_map(ctx, m)
        close(got, ref, tot["shot"], "parts")
        # served requests (FP32, FP64 and far-field waves)
        reqs = [mm.mm_submit(ctx, lh, mm.params(**CFG0, precision=p)) for p in (mm.MM_FP32C, mm.MM_FP64)] + \
               [mm.mm_submit(ctx, 0, mm.params(**SPLIT, nstar=2000, disc_radius=8.0)),
                mm.mm_submit(ctx, lb, mm.params(**SPLIT, precision=mm.MM_FAR32, far_ratio=0.05))]
        for r in reqs:
            h = mm.mm_wait(ctx, r, 120.0)
            mm.mm_release_map(ctx, h)
    finally:
        mm.mm_destroy(ctx)
    # the allocation-free entry point
    import torch
    dev = torch.device("cuda:0")
    x, y, w = (torch.from_numpy(a).to(dev) for a in (f.x, f.y, f.m))
    counts = torch.zeros(128 * 128, dtype=torch.int32, device=dev)
    totals = torch.zeros(2, dtype=torch.int64, device=dev)
    mm.mm_shoot_noalloc(x.data_ptr(), y.data_ptr(), w.data_ptr(), f.n, mm.params(**CFG0), counts.data_ptr(),
                        totals.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    close(counts.cpu().numpy().view(np.uint32).reshape(128, 128), ref, tot["shot"], "noalloc")
    print("checked build: every path ran without a failed bounds check")
    return 0


if __name__ == "__main__":
    sys.exit(main())
