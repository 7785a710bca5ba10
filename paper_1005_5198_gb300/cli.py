"""Command line: shoot a magnification map from a JSON description of its parameters.

    python -m paper_1005_5198_gb300.cli configs
    python -m paper_1005_5198_gb300.cli geometry --config fig1
    python -m paper_1005_5198_gb300.cli shoot --config fig1 --out fig1.npy [--stats fig1.json]
    python -m paper_1005_5198_gb300.cli shoot --config fig1 --out fig1.npy \\
        --parts 8 --checkpoint fig1.ckpt.npz [--max-parts-this-run 2]

    python -m paper_1005_5198_gb300.cli shoot --config fig1 --out fig1.npy --image fig1.png
    python -m paper_1005_5198_gb300.cli lightcurve --config fig1 --profile gaussian --size 0.05 \
        --start -8,0 --end 8,0 --points 2000 --out lc.npy

A config is a JSON object whose keys are mm_params field names (sigma, gamma, smooth_frac,
side_re, npix_side, nrays_per_pix, shoot_margin, nstar, disc_radius, mass_mu, mass_s, seed,
far_order, far_ratio, far_block, far_group_order, far_group_theta, far_group_leaf), plus precision ("fp32c", "fp64" or "far32"), mass_model
("unit" or "lognormal") and an optional "name"; --set key=value overrides one. A bare name
selects a config shipped in paper_1005_5198_gb300/configs. Lenses come from the seeded
generator (mm_create_lenses): N* and the disc follow Eq. nstar and the disc rule unless given.

--image writes the map as an 8-bit grayscale PNG of Delta m = -2.5 log10 mu (Sect. 3.1;
bright = magnified, clipped to the 1st..99th percentiles; pixels without a ray are black;
row J of the map, along y2, from the bottom). lightcurve shoots the map, convolves it with
a Gaussian or uniform-disc source of the given size (Einstein radii) and samples it along a
straight source track (Sect. 1), writing the magnifications as a float64 .npy array.

With --parts, the ray lattice is shot in bands of rows through mm_shoot_into. After each band
the counts and stats are written to the checkpoint (atomically); a run that finds the
checkpoint restores the map with mm_map_restore and goes on after its last band. The bands
start on the tile grid (on the block grid for far32), so the result is the one-shot map bit
for bit. --max-parts-this-run ends a run early (exit status 3) with the checkpoint written.
"""
from __future__ import annotations

import argparse
import json
import os
import struct
import sys
import zlib

import numpy as np

from . import (MM_FAR32, MM_FP32C, MM_FP64, MM_MASS_LOGNORMAL, MM_MASS_UNIT, MM_PROFILE_DISC, MM_PROFILE_GAUSSIAN,
               build, mm_destroy, mm_geometry_of, mm_init, mm_map_fetch, mm_map_lightcurve, mm_map_restore,
               mm_release_map, mm_shoot, mm_shoot_into, params)

CONFIG_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs")
PRECISIONS = {"fp32c": MM_FP32C, "fp64": MM_FP64, "far32": MM_FAR32}
MASS_MODELS = {"unit": MM_MASS_UNIT, "lognormal": MM_MASS_LOGNORMAL}
NUMERIC = {"sigma", "gamma", "smooth_frac", "side_re", "npix_side", "nrays_per_pix", "shoot_margin", "nstar",
           "disc_radius", "mass_mu", "mass_s", "seed", "far_order", "far_ratio", "far_block", "far_group_order",
           "far_group_theta", "far_group_leaf"}
INTEGER = {"npix_side", "nstar", "seed", "far_order", "far_block", "far_group_order", "far_group_leaf"}
EXIT_INTERRUPTED = 3


def shipped_configs() -> list[str]:
    return sorted(f[:-5] for f in os.listdir(CONFIG_DIR) if f.endswith(".json"))


def load_config(spec: str, overrides=()) -> dict:
    """The config named `spec` (shipped) or stored at path `spec`, with key=value overrides applied."""
    path = spec if os.path.exists(spec) else os.path.join(CONFIG_DIR, spec + ".json")
    if not os.path.exists(path):
        raise ValueError(f"no config {spec!r} (shipped: {', '.join(shipped_configs())})")
    with open(path) as fh:
        cfg = json.load(fh)
    for kv in overrides:
        k, _, v = kv.partition("=")
        cfg[k.strip()] = v.strip() if k.strip() in ("precision", "mass_model", "name") else float(v)
    unknown = set(cfg) - NUMERIC - {"precision", "mass_model", "name"}
    if unknown:
        raise ValueError(f"unknown config keys: {sorted(unknown)}")
    if cfg.get("precision", "fp32c") not in PRECISIONS:
        raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
    if cfg.get("mass_model", "unit") not in MASS_MODELS:
        raise ValueError(f"mass_model must be one of {sorted(MASS_MODELS)}")
    return cfg


def to_params(cfg: dict, ray_rect=None):
    kw = {k: (int(v) if k in INTEGER else float(v)) for k, v in cfg.items() if k in NUMERIC}
    kw["precision"] = PRECISIONS[cfg.get("precision", "fp32c")]
    kw["mass_model"] = MASS_MODELS[cfg.get("mass_model", "unit")]
    if ray_rect is not None:
        kw["ray_rect"] = ray_rect
    return params(**kw)


def band_plan(ny: int, parts: int, align: int) -> list[int]:
    """Row boundaries 0 = j_0 < j_1 < ... = ny of up to `parts` bands; inner ones multiples of align."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    cuts = [0]
    for k in range(1, parts):
        j = (k * ny // parts) // align * align
        if cuts[-1] < j < ny:
            cuts.append(j)
    cuts.append(ny)
    return cuts


def _canonical(cfg: dict) -> str:
    return json.dumps({k: v for k, v in cfg.items() if k != "name"}, sort_keys=True)


def _save_checkpoint(path, counts, stats, next_part, plan, cfg):
    tmp = path + ".tmp.npz"
    np.savez(tmp, counts=counts.ravel(), stats=json.dumps(stats), next_part=next_part, plan=np.asarray(plan),
             config=_canonical(cfg))
    os.replace(tmp, path)


def write_png(path: str, gray: np.ndarray) -> None:
    """An 8-bit grayscale PNG (colour type 0) of a 2-D uint8 array, first row at the top."""
    gray = np.ascontiguousarray(gray, dtype=np.uint8)
    h, w = gray.shape
    raw = b"".join(b"\x00" + gray[r].tobytes() for r in range(h))       # filter type 0 per row

    def chunk(tag, data):
        return struct.pack(">I", len(data)) + tag + data + struct.pack(">I", zlib.crc32(tag + data) & 0xFFFFFFFF)

    png = (b"\x89PNG\r\n\x1a\n" + chunk(b"IHDR", struct.pack(">IIBBBBB", w, h, 8, 0, 0, 0, 0)) +
           chunk(b"IDAT", zlib.compress(raw, 6)) + chunk(b"IEND", b""))
    with open(path, "wb") as fh:
        fh.write(png)


def delta_m_image(counts: np.ndarray, nrays: float) -> np.ndarray:
    """Grayscale of Delta m = -2.5 log10(N / N_rays): bright = magnified, clipped to the 1st..99th
    percentiles of the pixels with rays, black where no ray landed; map row J (y2) from the bottom."""
    mu = counts.astype(np.float64) / nrays
    img = np.zeros(counts.shape, dtype=np.uint8)
    lit = mu > 0
    if lit.any():
        dm = -2.5 * np.log10(mu[lit])
        lo, hi = np.percentile(dm, [1, 99])
        scale = (hi - np.clip(dm, lo, hi)) / max(hi - lo, 1e-12)       # 1 = most magnified
        img[lit] = (1 + np.round(254 * scale)).astype(np.uint8)
    return img[::-1]


def cmd_geometry(args):
    cfg = load_config(args.config, args.set)
    print(json.dumps(mm_geometry_of(to_params(cfg))))
    return 0


def cmd_shoot(args):
    cfg = load_config(args.config, args.set)
    p = to_params(cfg)
    g = mm_geometry_of(p)
    build()
    ctx = mm_init(args.device)
    try:
        if args.parts is None:
            m = mm_shoot(ctx, 0, p)
        else:
            align = 32 * (g["far_block"] if p.precision == MM_FAR32 else 1)
            plan = band_plan(g["ny"], args.parts, align)
            start = 0
            if args.checkpoint and os.path.exists(args.checkpoint):
                with np.load(args.checkpoint) as ck:
                    if str(ck["config"]) != _canonical(cfg) or list(ck["plan"]) != plan:
                        raise SystemExit(f"{args.checkpoint} belongs to another config or band plan")
                    m = mm_map_restore(ctx, 0, p, ck["counts"], json.loads(str(ck["stats"])))
                    start = int(ck["next_part"])
            else:
                m = mm_shoot(ctx, 0, to_params(cfg, ray_rect=(0, 0, 0, 0)))
            done = 0
            for k in range(start, len(plan) - 1):
                if args.max_parts_this_run is not None and done >= args.max_parts_this_run:
                    print(f"stopped after band {k} of {len(plan) - 1}; resume from {args.checkpoint}")
                    return EXIT_INTERRUPTED
                mm_shoot_into(ctx, 0, to_params(cfg, ray_rect=(0, g["nx"], plan[k], plan[k + 1])), m)
                done += 1
                if args.checkpoint:
                    counts, st = mm_map_fetch(ctx, m)
                    _save_checkpoint(args.checkpoint, counts, st, k + 1, plan, cfg)
        counts, st = mm_map_fetch(ctx, m)
        mm_release_map(ctx, m)
    finally:
        mm_destroy(ctx)
    np.save(args.out, counts)
    if args.image:
        write_png(args.image, delta_m_image(counts, p.nrays_per_pix))
    stats = dict(st, config=cfg.get("name", args.config), geometry=g)
    if args.stats:
        with open(args.stats, "w") as fh:
            json.dump(stats, fh, indent=1)
    print(json.dumps({k: stats[k] for k in ("rays_shot", "rays_in", "rays_out", "mu_mean", "seconds", "far_bound")}))
    return 0


def cmd_lightcurve(args):
    cfg = load_config(args.config, args.set)
    p = to_params(cfg)
    start = [float(v) for v in args.start.split(",")]
    end = [float(v) for v in args.end.split(",")]
    if len(start) != 2 or len(end) != 2:
        raise SystemExit("--start and --end take y1,y2 (Einstein radii)")
    profile = {"gaussian": MM_PROFILE_GAUSSIAN, "disc": MM_PROFILE_DISC}[args.profile]
    build()
    ctx = mm_init(args.device)
    try:
        m = mm_shoot(ctx, 0, p)
        lc = mm_map_lightcurve(ctx, m, profile, args.size, start, end, args.points)
        mm_release_map(ctx, m)
    finally:
        mm_destroy(ctx)
    np.save(args.out, lc)
    ok = lc[np.isfinite(lc)]
    print(json.dumps({"points": int(lc.size), "with_value": int(ok.size),
                      "mu_min": float(ok.min()) if ok.size else None, "mu_max": float(ok.max()) if ok.size else None}))
    return 0


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_1005_5198_gb300.cli", description=__doc__.split("\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    sub.add_parser("configs", help="list the shipped configs")
    for name in ("geometry", "shoot", "lightcurve"):
        sp = sub.add_parser(name)
        sp.add_argument("--config", required=True, help="shipped config name or JSON file")
        sp.add_argument("--set", action="append", default=[], metavar="KEY=VALUE", help="override a config key")
        if name == "lightcurve":
            sp.add_argument("--profile", choices=["gaussian", "disc"], default="gaussian")
            sp.add_argument("--size", type=float, required=True, help="source size (Einstein radii)")
            sp.add_argument("--start", required=True, help="track start y1,y2 (Einstein radii)")
            sp.add_argument("--end", required=True, help="track end y1,y2")
            sp.add_argument("--points", type=int, default=1000)
            sp.add_argument("--out", required=True, help="magnifications as a float64 .npy array")
            sp.add_argument("--device", type=int, default=0)
        if name == "shoot":
            sp.add_argument("--out", required=True, help="counts as a uint32 .npy array [N_side, N_side]")
            sp.add_argument("--image", help="also write the map as a grayscale PNG of Delta m")
            sp.add_argument("--stats", help="write the map's stats and geometry as JSON")
            sp.add_argument("--device", type=int, default=0)
            sp.add_argument("--parts", type=int, help="shoot in this many bands of ray rows")
            sp.add_argument("--checkpoint", help="checkpoint file for --parts (written after each band)")
            sp.add_argument("--max-parts-this-run", type=int, help="stop after this many bands (exit status 3)")
    args = ap.parse_args(argv)
    if args.cmd == "configs":
        for c in shipped_configs():
            print(f"{c}: {load_config(c).get('name', '')}")
        return 0
    return {"geometry": cmd_geometry, "shoot": cmd_shoot, "lightcurve": cmd_lightcurve}[args.cmd](args)


if __name__ == "__main__":
    sys.exit(main())
