"""Parameter sweeps of the paper's timing tests (Sect. 3.2, Figs. 2-4) on the GPU.

The paper times map generation against convergence (sigma = 0.1 .. 0.9, gamma = 0,
s = 0; Sect. 3.2.1), against shear (sigma = sigma_* = 0.45, gamma = 0 .. 1.0;
Sect. 3.2.2) and against the smooth-matter fraction (sigma = 0.45, gamma = 0.5,
s = 0 .. 0.9 and 0.99; Sect. 3.2.3), for source planes of side 20 Einstein radii
and N_rays = 1000. N* follows from the parameters (Eq. nstar with the disc rule of
the library). Each point is shot once through mm_shoot after a warm-up, with
the exact FP32 path (default), the plain FP64 kernel, or the far-field
approximation MM_FAR32 (the tree code's idea, default order, ratio and block),
and reported with N*, the theoretical mean magnification (Eq. mutheory), the
rays and interactions shot, the device time and the rate (for the far field:
the exact method's interactions per second of its own time, and its tail
bound). Points whose interaction count (far field: ray count) exceeds
--max-interactions (--max-rays) are listed but not shot.

    python -m paper_1005_5198_gb300.sweep --sweep sigma --npix 1024 --nrays 1000
    python -m paper_1005_5198_gb300.sweep --sweep sigma --npix 1024 --nrays 1000 --precision far32
"""
from __future__ import annotations

import argparse
import json
import math
import sys

import paper_1005_5198_gb300 as mm

SWEEPS = {
    "sigma": [dict(sigma=round(0.1 * k, 2), gamma=0.0, smooth_frac=0.0) for k in range(1, 10)],
    "gamma": [dict(sigma=0.45, gamma=round(0.1 * k, 2), smooth_frac=0.0) for k in range(0, 11)],
    "smooth": [dict(sigma=0.45, gamma=0.5, smooth_frac=round(0.1 * k, 2)) for k in range(0, 10)]
    + [dict(sigma=0.45, gamma=0.5, smooth_frac=0.99)],
}


PRECISIONS = {"fp32c": mm.MM_FP32C, "fp64": mm.MM_FP64, "far32": mm.MM_FAR32}


def plan(sweep: str, npix: int, nrays: float, side: float = 20.0, precision: str = "fp32c"):
    pts = []
    for q in SWEEPS[sweep]:
        p = mm.params(**q, side=side, npix_side=npix, nrays=nrays, precision=PRECISIONS[precision])
        try:
            g = mm.mm_geometry_of(p)
        except mm.MMError as e:                 # ill-posed (|1 - sigma -+ gamma| < 1e-3)
            pts.append(dict(q, error=str(e)))
            continue
        pts.append(dict(q, nstar=g["nstar"], mu_av=g["mu_theory"], rays=g["nx"] * g["ny"],
                        interactions=g["nx"] * g["ny"] * g["nstar"], params=p))
    return pts


def run(sweep: str, npix: int, nrays: float, max_interactions: float, device: int = 0, precision: str = "fp32c",
        max_rays: float = 2e12, compare_exact: bool = False, keep_counts: bool = False):
    """Shoot every point of a sweep; one row per point (keep_counts: each row also holds the map's
    uint32 counts, [N_side, N_side])."""
    mm.build()
    ctx = mm.mm_init(device)
    out = []
    try:
        warm = mm.mm_shoot(ctx, 0, mm.params(sigma=0.4, gamma=0.0, side=4.0, npix_side=64, nrays=10.0, nstar=100,
                                             precision=PRECISIONS[precision]))
        mm.mm_release_map(ctx, warm)
        for pt in plan(sweep, npix, nrays, precision=precision):
            row = {k: v for k, v in pt.items() if k != "params"}
            if "error" in pt:
                out.append(row)
                continue
            if precision != "far32" and pt["interactions"] > max_interactions:
                row["skipped"] = f"{pt['interactions']:.2e} interactions above the cap"
                out.append(row)
                continue
            if precision == "far32" and pt["rays"] > max_rays:
                row["skipped"] = f"{pt['rays']:.2e} rays above the cap"
                out.append(row)
                continue
            m = mm.mm_shoot(ctx, 0, pt["params"])
            ms, _ = mm.mm_last_kernel_ms(ctx)
            counts, st = mm.mm_map_fetch(ctx, m, want_counts=keep_counts)
            if keep_counts:
                row["counts"] = counts.copy()
            if compare_exact and pt["interactions"] <= max_interactions:
                # the paper's map statistics (Sect. 3.1) against the exact FP32 map of the same lenses
                q = pt["params"]
                q.precision = mm.MM_FP32C
                ex = mm.mm_shoot(ctx, 0, q)
                row["exact_ms"] = mm.mm_last_kernel_ms(ctx)[0]
                cmp = mm.mm_map_compare(ctx, m, ex)
                row.update(rms_dm_vs_exact=cmp["rms_dm"], ks_p_vs_exact=cmp["ks_p"], ks_d_vs_exact=cmp["ks_d"])
                mm.mm_release_map(ctx, ex)
            mm.mm_release_map(ctx, m)
            row.update(kernel_ms=ms, interactions_per_s=st["interactions"] / (ms * 1e-3) if ms > 0 else None,
                       mu_map=st["mu_mean"], lens_splits=st["lens_splits"], far_bound=st["far_bound"],
                       rays_shot=st["rays_shot"], rays_in=st["rays_in"], rays_out=st["rays_out"])
            out.append(row)
    finally:
        mm.mm_destroy(ctx)
    return out


def compare_table(rows, sweep, npix, nrays):
    head = (f"Sweep `{sweep}`, N_pix = {npix}^2, N_rays = {nrays:g}, L = 20 R_E: far field against the exact FP32 "
            "map of the same lenses (Sect. 3.1 statistics)\n\n"
            "| sigma | gamma | s | N* | far ms | exact ms | speed-up | bound (R_E) | RMS delta-m (mag) | K-S D | "
            "K-S probability |\n|---|---|---|---|---|---|---|---|---|---|---|\n")
    lines = []
    for r in rows:
        if "rms_dm_vs_exact" not in r:
            continue
        lines.append(f"| {r['sigma']} | {r['gamma']} | {r['smooth_frac']} | {r['nstar']} | {r['kernel_ms']:.1f} | "
                     f"{r['exact_ms']:.1f} | {r['exact_ms'] / r['kernel_ms']:.1f}x | {r['far_bound']:.1g} | "
                     f"{r['rms_dm_vs_exact']:.2e} | {r['ks_d_vs_exact']:.2e} | {r['ks_p_vs_exact']:.4f} |")
    return head + "\n".join(lines) + "\n"


def table(rows, sweep, npix, nrays, precision="fp32c"):
    path = {"fp32c": "FP32 path", "fp64": "plain FP64 kernel",
            "far32": "far field MM_FAR32, rate in exact-method interactions per second; bound in R_E"}[precision]
    head = (f"Sweep `{sweep}`, N_pix = {npix}^2, N_rays = {nrays:g}, L = 20 R_E ({path}, one map per point)\n\n"
            "| sigma | gamma | s | N* | mu_av (Eq. mutheory) | rays | interactions | GPU ms | interactions/s |"
            + (" bound |" if precision == "far32" else "") + "\n"
            "|---|---|---|---|---|---|---|---|---|" + ("---|" if precision == "far32" else "") + "\n")
    lines = []
    for r in rows:
        base = f"| {r['sigma']} | {r['gamma']} | {r['smooth_frac']} |"
        if "error" in r:
            lines.append(base + " - | - | - | - | ill-posed | |")
        elif "skipped" in r:
            lines.append(base + f" {r['nstar']} | {r['mu_av']:.3g} | {r['rays']:.3g} | {r['interactions']:.3g} | "
                                f"not shot ({r['skipped']}) | |")
        else:
            lines.append(base + f" {r['nstar']} | {r['mu_av']:.3g} | {r['rays']:.3g} | {r['interactions']:.3g} | "
                                f"{r['kernel_ms']:.1f} | {r['interactions_per_s']:.3g} |"
                         + (f" {r['far_bound']:.2g} |" if precision == "far32" else ""))
    return head + "\n".join(lines) + "\n"


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--sweep", choices=sorted(SWEEPS), required=True)
    ap.add_argument("--npix", type=int, default=1024, help="N_side (the paper: 1024, 2048, 4096)")
    ap.add_argument("--nrays", type=float, default=1000.0, help="N_rays (the paper: 1000)")
    ap.add_argument("--max-interactions", type=float, default=2e14)
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="fp32c")
    ap.add_argument("--max-rays", type=float, default=2e12, help="far field: skip points with more rays")
    ap.add_argument("--compare-exact", action="store_true",
                    help="far field: also shoot the exact FP32 map of each point (up to --max-interactions) and "
                         "report the paper's map statistics between the two")
    ap.add_argument("--json", action="store_true", help="print JSON lines instead of a table")
    a = ap.parse_args(argv)
    if a.compare_exact and a.precision != "far32":
        raise SystemExit("--compare-exact needs --precision far32")
    rows = run(a.sweep, a.npix, a.nrays, a.max_interactions, precision=a.precision, max_rays=a.max_rays,
               compare_exact=a.compare_exact)
    if a.json:
        for r in rows:
            print(json.dumps(r))
    else:
        sys.stdout.write(table(rows, a.sweep, a.npix, a.nrays, a.precision))
        if a.compare_exact:
            sys.stdout.write("\n" + compare_table(rows, a.sweep, a.npix, a.nrays))
    return 0


if __name__ == "__main__":
    sys.exit(main())
