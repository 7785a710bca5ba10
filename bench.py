"""Benchmark: direct inverse ray-shooting of the Fig. 1 map on one GB300.

One step = one complete magnification map through the library's C ABI: the
whole hot path (ray lattice, deflection sum over all N* lenses, lens-equation
epilogue, binning) for the Fig. 1 workload -- sigma = 0.4, gamma = 0, L = 20
Einstein radii, N_side = 1024, N_rays = 2000, N* = 558 unit lenses (1.31e10
rays, 7.31e12 ray-lens interactions) -- with the lens set resident in HBM.

Reported (one JSON line from rank 0):
  value        ray-lens interactions / s, FP32 compensated path, whole job
  e2e          the same through the public API with host buffers: lens arrays
               uploaded from pinned memory, map shot, counts read back, per step
  roofline     the shoot kernel against the FP32 ALU peak (the device's SMs x
               128 lanes x 2 FLOP x 2070 MHz), algorithmic FLOP = 10 per
               interaction (the paper's N_FLOP convention for the deflection of
               one ray by one lens); also against the measured FFMA rate
  fp64         the plain FP64 kernel on a ray window of the same map
  cpu_baseline the FP64 CPU oracle on a strided sample of the same map
  clocks       nvidia-smi samples taken during the timed region

--impl reference times the CPU oracle (the reference arm of this build).
Multi-GPU (torchrun): every rank shoots its own map (independent problems, no
collective), value = total interactions / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CFG1 = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=20.0, npix_side=1024, nrays=2000.0)
SEED = 2
FLOP_PER_INTERACTION = 10.0      # Eq. for Phi: N_FLOP = 10 per deflection evaluation
USEFUL_OPS_PER_INTERACTION = 6.0  # FP32 lane operations no implementation avoids: 2 sub, 1 mul, 3 fma
USEFUL_OPS_WITH_MASSES = 7.0      # the same plus the mass product, for maps with a mass spectrum
LANES, SM_MAX_MHZ = 128, 2070.0
# FFMA lane operations per SM per clock measured on GB300 by the pipe probe (bench.py --alu-rates,
# alu_rates.cu): the attainable FP32 rate, slightly under the 128 lanes of the data sheet
FFMA_MEASURED_LANE_OPS = 125.1


def fp32_peak_tflops(sms: int, lane_ops: float = LANES) -> float:
    """FP32 FLOP peak: SMs x lane operations per clock x 2 FLOP (FMA) x the maximum SM clock."""
    return sms * lane_ops * 2 * SM_MAX_MHZ * 1e6 / 1e12


def lane_peak_per_s(sms: int) -> float:
    """FP32 lane operations per second at the maximum SM clock."""
    return sms * LANES * SM_MAX_MHZ * 1e6


def device_sms(device: int) -> int:
    import torch
    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def lens_rule(mm, p):
    """N* and disc radius of a map from the library's own rule (Eq. nstar with the disc reading)."""
    g = mm.mm_geometry_of(p)
    return int(g["nstar"]), float(g["disc_radius"])
WORKLOAD = ("Fig. 1 map: sigma=0.4, gamma=0, s=0, L=20 R_E, N_pix=1024^2, N_rays=2000, N*=558 unit masses "
            "uniform in a disc of R=37.36 R_E (seed 2); 114487^2 = 1.31e10 rays")
METRIC = "ray-lens interactions/s and maps/s on 1 GB300 (FP32 vs FP64); p50/p99 map latency"
CPU_STRIDE = 12                   # oracle sample: every 12th ray row and column (1/144 of the rays)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class Clocks:
    """nvidia-smi sampler for the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, directory: str | None = None):
        import tempfile
        self.device = device
        self.proc = None
        self.path = os.path.join(directory or tempfile.gettempdir(), f"clocks_rank{device}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


def scaled_mix(count, seed, sides=(64, 128, 256), nrays=(10.0, 30.0, 100.0), cap=4e11, large_every=0):
    """Map requests with the config-3 parameter distributions (sigma, gamma, s, L, lognormal masses),
    scaled down in N_side and N_rays so that a phase fits in seconds; maps above `cap` interactions
    are redrawn. Every `large_every`-th request is 4x the pixels (the "large" share of config 4)."""
    import paper_1005_5198_gb300 as mm
    import synth
    out, k = [], 0
    while len(out) < count:
        k += 1
        d = synth.map_mix(1, seed * 1000003 + k, sides=sides, nrays=nrays)[0]
        large = bool(large_every) and (len(out) % large_every == large_every - 1)
        nside = d.npix_side * (2 if large else 1)
        p = mm.params(sigma=d.sigma, gamma=d.gamma, smooth_frac=d.smooth_frac, side=d.side, npix_side=nside,
                      nrays=d.nrays, mass_model=mm.MM_MASS_LOGNORMAL, mass_s=0.5, seed=d.seed)
        g = mm.mm_geometry_of(p)
        inter = g["nx"] * g["ny"] * g["nstar"]
        if inter > cap * (4 if large else 1) or g["nstar"] == 0:
            continue
        out.append((p, inter))
    return out


def scaled_batch_phase(mm, ctx, sms, n_maps=64, seed=4):
    """Secondary line: the config-3 parameter mix scaled down (N_side in {64, 128, 256}, N_rays in
    {10, 30, 100}, maps above 4e11 interactions redrawn) in ONE persistent launch, best of 3."""
    mix = scaled_mix(n_maps, seed)
    plist = [p for p, _ in mix]
    total = sum(i for _, i in mix)
    maps = mm.mm_shoot_batch(ctx, None, plist)          # warm-up (and lens generation)
    for m in maps:
        mm.mm_release_map(ctx, m)
    t = []
    for _ in range(3):
        maps = mm.mm_shoot_batch(ctx, None, plist)
        t.append(mm.mm_last_kernel_ms(ctx)[0])
        for m in maps:
            mm.mm_release_map(ctx, m)
    batch_ms = min(t)
    return {"workload": f"{n_maps} maps, config-3 parameter mix (lognormal masses) scaled to N_side in "
                        "{64,128,256}, N_rays in {10,30,100}, <= 4e11 interactions each",
            "interactions": total, "batched_ms": batch_ms, "batched_interactions_per_s": total / (batch_ms * 1e-3),
            "maps_per_s": n_maps / (batch_ms * 1e-3)}


CFG2 = dict(sigma=0.8, gamma=0.3, smooth_frac=0.5, side=40.0, npix_side=2048, nrays=500.0)
CFG2_NSTAR, CFG2_SEED = 25000, 3


def config2_phase(mm, ctx, sms, band_fraction=16):
    """The exact FP32 path on the high-optical-depth map (sigma = 0.8, s = 0.5, gamma = 0.3, L = 40,
    2048^2 pixels, N_rays = 500, N* = 25000 unit lenses in a disc of 250 R_E, seed 3): the central
    band of 1/band_fraction of the ray rows across the whole width of the 686921 x 137385-ray grid
    (600 x 120 R_E), one mm_shoot with that ray_rect, timed by CUDA events (mm_last_kernel_ms)."""
    import synth
    p0 = mm.params(**CFG2, nstar=CFG2_NSTAR)
    g = mm.mm_geometry_of(p0)
    f = synth.lens_field(int(g["nstar"]), float(g["disc_radius"]), CFG2_SEED)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    h = g["ny"] // (2 * band_fraction)
    rect = (0, g["nx"], g["ny"] // 2 - h, g["ny"] // 2 + h)
    p = mm.params(**CFG2, nstar=CFG2_NSTAR, ray_rect=rect)
    m = mm.mm_shoot(ctx, lh, p)
    ms, _ = mm.mm_last_kernel_ms(ctx)
    _, st = mm.mm_map_fetch(ctx, m, want_counts=False)
    mm.mm_release_map(ctx, m)
    mm.mm_release_lenses(ctx, lh)
    rate = st["interactions"] / (ms * 1e-3)
    return {"workload": f"sigma=0.8, s=0.5, gamma=0.3, L=40 R_E, 2048^2 px, N_rays=500, N*=25000 unit masses "
                        f"(R=250 R_E, seed 3): ray rows [{rect[2]}, {rect[3]}) of {g['ny']} (1/{band_fraction} of the "
                        f"grid, full width {g['nx']})",
            "rays": st["rays_shot"], "interactions": st["interactions"], "ms": ms,
            "interactions_per_s": rate,
            "frac_nflop10": FLOP_PER_INTERACTION * rate / (fp32_peak_tflops(sms) * 1e12),
            "useful_frac": USEFUL_OPS_PER_INTERACTION * rate / lane_peak_per_s(sms),
            "whole_map_estimated_s": g["nx"] * g["ny"] * g["nstar"] / rate,
            "lens_splits": st["lens_splits"]}


CFG3_SIDES, CFG3_NRAYS, CFG3_CAP = (256, 512, 1024), (100.0, 300.0, 1000.0), 5e13


def config3_phase(mm, ctx, sms, n_maps=64, seed=4, fp64_interactions_per_map=6e9):
    """The batched pattern on its own workload: 64 maps with sigma ~ U(0.2, 1.5), gamma ~ U(0, 0.6),
    s ~ U(0, 0.9), L ~ U(10, 40) R_E, N_side in {256, 512, 1024}, N_rays in {100, 300, 1000},
    lognormal(0, 0.5) masses, N* by the library's rule with <M> = e^0.125 (seeded; draws with
    min |1 - sigma -+ gamma| < 0.05 redrawn, and maps above 5e13 interactions redrawn: the capped
    variant, about 4.4e14 interactions in all). Lens sets are made first; then the 64 maps in ONE
    persistent launch (mm_shoot_batch, timed by CUDA events), the same maps one by one (mm_shoot),
    a bit-identity check of batched against alone on 8 maps, and the plain FP64 kernel one map at a
    time on a central band of each map's ray rows holding about 6e9 interactions."""
    mix = scaled_mix(n_maps, seed, sides=CFG3_SIDES, nrays=CFG3_NRAYS, cap=CFG3_CAP)
    plist = [p for p, _ in mix]
    total = sum(i for _, i in mix)
    lenses = [mm.mm_create_lenses(ctx, p) for p in plist]
    small = sorted(range(n_maps), key=lambda k: mix[k][1])[:4]
    warm = mm.mm_shoot_batch(ctx, [lenses[k] for k in small], [plist[k] for k in small])   # kernels warm
    for m in warm:
        mm.mm_release_map(ctx, m)
    batched = mm.mm_shoot_batch(ctx, lenses, plist)
    batch_ms = mm.mm_last_kernel_ms(ctx)[0]
    one_ms, identical, checked = 0.0, 0, 0
    check = set(sorted(range(n_maps), key=lambda k: mix[k][1])[::8])        # 8 maps across the sizes
    for k, p in enumerate(plist):
        m = mm.mm_shoot(ctx, lenses[k], p)
        one_ms += mm.mm_last_kernel_ms(ctx)[0]
        if k in check:
            a, _ = mm.mm_map_fetch(ctx, m)
            b, _ = mm.mm_map_fetch(ctx, batched[k])
            identical += int(np.array_equal(a, b))
            checked += 1
        mm.mm_release_map(ctx, m)
    for m in batched:
        mm.mm_release_map(ctx, m)
    f64_ms, f64_inter = 0.0, 0
    for k, p in enumerate(plist):
        g = mm.mm_geometry_of(p)
        rows = max(1, min(g["ny"], int(fp64_interactions_per_map / max(1, g["nx"] * g["nstar"]))))
        q = mm.params(**{f: getattr(p, f) for f, _ in mm.mm_params._fields_ if f != "ray_rect"})
        q.precision = mm.MM_FP64
        q.ray_rect[:] = [0, g["nx"], g["ny"] // 2 - rows // 2, g["ny"] // 2 - rows // 2 + rows]
        m = mm.mm_shoot(ctx, lenses[k], q)
        f64_ms += mm.mm_last_kernel_ms(ctx)[0]
        _, st = mm.mm_map_fetch(ctx, m, want_counts=False)
        f64_inter += st["interactions"]
        mm.mm_release_map(ctx, m)
    for h in lenses:
        mm.mm_release_lenses(ctx, h)
    rate = total / (batch_ms * 1e-3)
    inters = sorted(i for _, i in mix)
    return {"workload": f"{n_maps} maps of the config-3 mix: sigma~U(0.2,1.5), gamma~U(0,0.6), s~U(0,0.9), "
                        "L~U(10,40) R_E, N_side in {256,512,1024}, N_rays in {100,300,1000}, lognormal(0,0.5) "
                        "masses, seed 4; maps above 5e13 interactions redrawn (capped variant)",
            "interactions": total, "interactions_median": inters[len(inters) // 2], "interactions_max": inters[-1],
            "nstar_max": max(int(mm.mm_geometry_of(p)["nstar"]) for p in plist),
            "batched_ms": batch_ms, "batched_interactions_per_s": rate, "maps_per_s": n_maps / (batch_ms * 1e-3),
            "frac_nflop10": FLOP_PER_INTERACTION * rate / (fp32_peak_tflops(sms) * 1e12),
            "useful_frac": USEFUL_OPS_WITH_MASSES * rate / lane_peak_per_s(sms),
            "one_by_one_ms": one_ms, "one_by_one_interactions_per_s": total / (one_ms * 1e-3),
            "one_by_one_maps_per_s": n_maps / (one_ms * 1e-3),
            "batched_identical_to_alone": f"{identical} of {checked} maps bit-identical",
            "fp64_one_by_one_interactions_per_s": f64_inter / (f64_ms * 1e-3),
            "fp64_sample": f"plain FP64 kernel, each of the {n_maps} maps on a central band of its ray rows "
                           f"(about {fp64_interactions_per_map:.0e} interactions per map, {f64_inter:.3e} in all)",
            "fp32_batched_over_fp64": rate / (f64_inter / (f64_ms * 1e-3))}


def config4_stream(count, seed, large_every=10, cap=CFG3_CAP, large_cap=2e14):
    """Requests of the served workload: the config-3 mix (capped at 5e13 interactions) with every
    large_every-th request "large": 2048^2 pixels and N* = 20000 lognormal lenses in the disc that
    Eq. nstar gives for kappa_* = sigma_*, its other parameters from the mix (redrawn above 2e14
    interactions)."""
    import paper_1005_5198_gb300 as mm
    import synth
    out, k = [], 0
    while len(out) < count:
        k += 1
        d = synth.map_mix(1, seed * 1000003 + k, sides=CFG3_SIDES, nrays=CFG3_NRAYS)[0]
        large = large_every and len(out) % large_every == large_every - 1
        kw = dict(sigma=d.sigma, gamma=d.gamma, smooth_frac=d.smooth_frac, side=d.side, nrays=d.nrays,
                  mass_model=mm.MM_MASS_LOGNORMAL, mass_s=0.5, seed=d.seed)
        p = mm.params(**kw, npix_side=2048, nstar=20000) if large else mm.params(**kw, npix_side=d.npix_side)
        g = mm.mm_geometry_of(p)
        inter = g["nx"] * g["ny"] * g["nstar"]
        if inter > (large_cap if large else cap) or g["nstar"] == 0:
            continue
        out.append((p, inter, bool(large)))
    return out


def config4_phase(mm, ctx, capacity, args, overload_s=45.0, load_s=90.0, drain_s=45.0):
    """The served workload (config 4): (i) the stated Poisson stream, lambda = 20 requests/s for 200
    arrivals, about 70x one GPU's capacity: observed for overload_s after the first arrival, then the
    rest is cancelled; (ii) lambda scaled to 70 % of the capacity measured by the batched launch on
    the config-3 maps, arrivals for load_s, then up to drain_s for the last ones. HBM-budgeted
    admission, device-resident lens sets and maps, waves of continuous batching."""
    import synth
    mm.mm_serve_config(ctx, max_active=64, wave_ms=args.wave_ms)
    mm.mm_serve_priority(ctx, args.serve_priority)
    sample = config4_stream(400, 6)
    mean_inter = float(np.mean([i for _, i, _ in sample]))
    over = config4_stream(200, 8)
    res_over = serve_phase(mm, ctx, over, synth.poisson_arrivals(200, 20.0, 8), overload_s, 0.0)
    lam = 0.7 * capacity / mean_inter
    n70 = max(8, int(round(lam * load_s)))
    load = config4_stream(n70, 7)
    res_70 = serve_phase(mm, ctx, load, synth.poisson_arrivals(n70, lam, 7), 0.0, drain_s)
    return {"workload": "config-4 stream: Poisson arrivals of the config-3 mix (capped at 5e13 interactions) "
                        "with every 10th request large (2048^2 px, N*=20000 lognormal lenses, kappa_*=sigma_*, "
                        "capped at 2e14); mm_submit/mm_poll continuous batching, latency from submit to completion",
            "capacity_interactions_per_s": capacity, "mean_request_interactions": mean_inter,
            "wave_ms": args.wave_ms, "priority_share": args.serve_priority,
            "overload_lambda_20": dict(res_over, lambda_req_s=20.0, observed_s=overload_s),
            "at_70pct_capacity": dict(res_70, lambda_req_s=lam)}


def serve_phase(mm, ctx, stream, arrivals, observe_s, drain_s):
    """Submit `stream` at the given arrival times (mm_submit), poll completions (mm_poll) until all
    are done or `observe_s` after the first arrival plus up to `drain_s` after the last arrival,
    then cancel what is left (mm_cancel) and wait for it. Latency = submit to completion (host
    clock, mm_req_times). Requests not done at the end enter the censored percentiles with their
    age at that moment (a lower bound of their latency). Device throughput = interactions of the
    work items shot during the run (mm_serve_stats) / run time."""
    import threading
    n = len(stream)
    reqs = [None] * n
    t_sub = [None] * n
    s0 = mm.mm_serve_stats(ctx)
    t0 = time.perf_counter()

    def submitter():
        for k in range(n):
            dt = arrivals[k] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            t_sub[k] = time.perf_counter()
            reqs[k] = mm.mm_submit(ctx, 0, stream[k][0])

    th = threading.Thread(target=submitter)
    th.start()
    end = max(observe_s, arrivals[-1] + drain_s)
    done = [False] * n
    lat = [None] * n
    finished = 0
    while finished < n and time.perf_counter() - t0 < end:
        progressed = False
        for k in range(n):
            if done[k] or reqs[k] is None:
                continue
            ok, m = mm.mm_poll(ctx, reqs[k])
            if ok:
                done[k] = True
                finished += 1
                progressed = True
                lat[k] = mm.mm_req_times(ctx, reqs[k])[1]
                mm.mm_release_map(ctx, m)
        if not progressed:
            time.sleep(0.005)        # latency comes from the server's own clock, not this loop's
    th.join()
    t_end = time.perf_counter()
    s1 = mm.mm_serve_stats(ctx)
    wall = t_end - t0
    cancelled = 0
    for k in range(n):
        if done[k]:
            continue
        try:
            mm.mm_cancel(ctx, reqs[k])
            cancelled += 1
        except mm.MMError:
            pass
    for k in range(n):                                   # wait for the rest to end (cancelled or done)
        if done[k]:
            continue
        try:
            m = mm.mm_wait(ctx, reqs[k], timeout_s=600)
            mm.mm_release_map(ctx, m)
        except mm.MMError as e:
            if e.code != mm.MM_ECANCELED:
                raise
    lat_done = np.array([x for x in lat if x is not None]) * 1e3
    censored = np.array([lat[k] * 1e3 if lat[k] is not None else (t_end - t_sub[k]) * 1e3 for k in range(n)])
    pct = (lambda a, q: float(np.percentile(a, q)) if len(a) else None)
    large_done = [lat[k] * 1e3 for k in range(n) if lat[k] is not None and stream[k][2]]
    return {"requests": n, "completed": int(len(lat_done)), "cancelled_at_end": cancelled,
            "large_requests": int(sum(1 for x in stream if x[2])), "large_completed": len(large_done),
            "p50_ms": pct(lat_done, 50), "p99_ms": pct(lat_done, 99), "max_ms": pct(lat_done, 100),
            "censored_p50_ms": pct(censored, 50), "censored_p99_ms": pct(censored, 99),
            "offered_interactions_per_s": sum(x[1] for x in stream) / max(arrivals[-1], 1e-9),
            "sustained_interactions_per_s": (s1["interactions"] - s0["interactions"]) / wall,
            "completed_interactions_per_s": sum(stream[k][1] for k in range(n) if done[k]) / wall,
            "wall_s": wall}


KERNEL_SOURCES = ["mm_fp32.cuh", "mm_device.cuh", "mm_internal.h", "mm_fp32_c2r4.cu"]


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of this GPU type (MEASURED_PEAKS.json), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def downstream_phase(mm, ctx, side=8192, fma_peak_per_s=None):
    """The rows after the map, on two side^2 maps (256 MiB of counts each at 8192^2, more than L2) of
    the Fig. 1 field at N_rays = 10, shot with the far field (default order and order 14):
    - the map statistics of Sect. 3.1 (mm_map_compare: RMS of Delta m and the K-S test), host clock
      around the call; algorithmic bytes: both maps read once (8 B/pixel);
    - the extended-source magnification maps (mm_map_convolve with a Gaussian or disc profile):
      device time of the convolution kernels (CUDA events, mm_last_kernel_ms); algorithmic bytes: the
      Gaussian's two separable passes read and write a map each (16 B/pixel), the disc reads the
      counts and writes the convolved map (8 B/pixel);
    - light curves along a track (mm_map_lightcurve, 1000 samples), which convolve only the four
      pixels around each sample: host clock around the call and the device time of its kernel.
    Each is the best of 3 after one warm-up."""
    peak, peak_src = hbm_peak_gbs()
    base = dict(sigma=0.4, gamma=0.0, smooth_frac=0.0, side=20.0, npix_side=side, nrays=10.0, seed=SEED)
    pa = mm.params(**base, precision=mm.MM_FAR32)
    pb = mm.params(**base, precision=mm.MM_FAR32, far_order=14)
    lh = mm.mm_create_lenses(ctx, pa)
    ma, mb = mm.mm_shoot(ctx, lh, pa), mm.mm_shoot(ctx, lh, pb)
    npix = side * side
    pix_re = 20.0 / side

    def timed(fn):
        """Best host time and best device time (mm_last_kernel_ms) of fn over 3 calls after a warm-up."""
        fn()
        best, best_dev, res = 1e30, 1e30, None
        for _ in range(3):
            t0 = time.perf_counter()
            res = fn()
            best = min(best, time.perf_counter() - t0)
            best_dev = min(best_dev, mm.mm_last_kernel_ms(ctx)[0] * 1e-3)
        return best, best_dev, res

    def line(sec, nbytes, extra):
        gbs = nbytes / sec / 1e9
        return dict(extra, ms=sec * 1e3, pixels_per_s=npix / sec, algorithmic_bytes=nbytes, achieved_gbs=gbs,
                    hbm_frac=gbs / peak)

    t_cmp, _, st = timed(lambda: mm.mm_map_compare(ctx, ma, mb))
    track = ((-8.0, -3.0), (8.0, 3.0))
    g_size, d_size = 0.02, 0.02
    h = int(np.ceil(4.0 * g_size / pix_re))
    hd = int(d_size / pix_re)
    _, k_cg, _ = timed(lambda: mm.mm_map_convolve(ctx, ma, mm.MM_PROFILE_GAUSSIAN, g_size))
    _, k_cd, _ = timed(lambda: mm.mm_map_convolve(ctx, ma, mm.MM_PROFILE_DISC, d_size))
    t_g, k_g, _ = timed(lambda: mm.mm_map_lightcurve(ctx, ma, mm.MM_PROFILE_GAUSSIAN, g_size, *track, 1000))
    t_d, k_d, _ = timed(lambda: mm.mm_map_lightcurve(ctx, ma, mm.MM_PROFILE_DISC, d_size, *track, 1000))
    route = "the four pixels around each sample, one CTA per sample (less work than the whole map)"
    out = {"workload": f"two {side}^2 maps of the Fig. 1 field (N_rays = 10, far field), {npix:.3e} pixels each",
           "hbm_peak_gbs": peak, "hbm_peak_source": peak_src,
           "compare": line(t_cmp, 8 * npix, {"rms_dm": st["rms_dm"], "ks_p": st["ks_p"]}),
           "convolve_gaussian": line(k_cg, 16 * npix, {"size_re": g_size, "taps_per_pass": 2 * h + 1,
                                                        "time": "device time of the two passes",
                                                        # the two passes' FMAs (one per tap and output)
                                                        # against the FP32 FMA peak: this kernel pair is
                                                        # bound by arithmetic before memory
                                                        "fma_frac": 2 * (2 * h + 1) * npix / k_cg
                                                                    / (fma_peak_per_s or 1.0)}),
           "convolve_disc": line(k_cd, 8 * npix, {"size_re": d_size, "radius_pixels": hd,
                                                  "time": "device time of the disc kernel"}),
           "lightcurve_gaussian": {"size_re": g_size, "taps_per_pass": 2 * h + 1, "points": 1000, "route": route,
                                   "ms": t_g * 1e3, "kernel_ms": k_g * 1e3},
           "lightcurve_disc": {"size_re": d_size, "radius_pixels": hd, "points": 1000, "route": route,
                               "ms": t_d * 1e3, "kernel_ms": k_d * 1e3}}
    mm.mm_release_map(ctx, ma)
    mm.mm_release_map(ctx, mb)
    mm.mm_release_lenses(ctx, lh)
    return out


def random_phase(mm, ctx, lh_fig1, exact_ms, sms):
    """Random rays (MM_RAYS_RANDOM: the paper's GPU code shoots rays from pseudo-random positions,
    Sect. 2.3 step 2) on the Fig. 1 map: the exact FP32 path at the same ray count as the lattice,
    timed like the headline (device time of the shoot, best of 3), and the paper's comparison of the
    random-ray map with the regular-grid map (Sect. 3.1: RMS of Delta m, K-S probability) made on the
    device by mm_map_compare."""
    p_lat = mm.params(**CFG1)
    p_rnd = mm.params(**CFG1, ray_mode=mm.MM_RAYS_RANDOM, ray_seed=SEED)
    best, m_rnd, st = 1e30, None, None
    for _ in range(3):
        if m_rnd:
            mm.mm_release_map(ctx, m_rnd)
        m_rnd = mm.mm_shoot(ctx, lh_fig1, p_rnd)
        kms, _ = mm.mm_last_kernel_ms(ctx)
        best = min(best, kms)
    _, st = mm.mm_map_fetch(ctx, m_rnd, want_counts=False)
    m_lat = mm.mm_shoot(ctx, lh_fig1, p_lat)
    cmp = mm.mm_map_compare(ctx, m_lat, m_rnd)
    for m in (m_lat, m_rnd):
        mm.mm_release_map(ctx, m)
    rate = st["interactions"] / (best * 1e-3)
    return {"workload": WORKLOAD + ", rays at random positions (each uniform in its 64 x 32-cell tile)",
            "ms": best, "interactions_per_s": rate, "vs_lattice_time": best / exact_ms,
            "frac_nflop10": FLOP_PER_INTERACTION * rate / 1e12 / fp32_peak_tflops(sms),
            "rays_in": st["rays_in"], "rays_shot": st["rays_shot"],
            "vs_lattice_rms_delta_m": cmp["rms_dm"], "vs_lattice_ks_probability": cmp["ks_p"],
            "excellent_agreement": bool(cmp["rms_dm"] < 0.2 and cmp["ks_p"] > 0.997)}


def far_phase(mm, ctx, lh_fig1, exact_ms):
    """The far-field approximation MM_FAR32 (the tree code's idea, Sect. 2.1; the library's default
    order, ratio and block), timed outside the headline region: the Fig. 1 map against the
    exact FP32 map of the same lenses, and the sigma = 0.8, N* = 25000 map (600 x 120 R_E shot
    region, 9.4e10 rays), whose exact shoot would take interactions / (the headline rate)."""
    import synth
    d = mm.params()
    out = {"params": {"far_order": d.far_order, "far_ratio": d.far_ratio, "far_block": d.far_block},
           "timing": "CUDA events around block preparation + shoot (mm_last_kernel_ms), best of 3"}
    m_ex = mm.mm_shoot(ctx, lh_fig1, mm.params(**CFG1))
    ex, st_ex = mm.mm_map_fetch(ctx, m_ex)
    ex = ex.copy()
    times = []
    for k in range(3):
        m = mm.mm_shoot(ctx, lh_fig1, mm.params(**CFG1, precision=mm.MM_FAR32))
        times.append(mm.mm_last_kernel_ms(ctx)[0])
        far, st = mm.mm_map_fetch(ctx, m)
        if k < 2:
            mm.mm_release_map(ctx, m)
    cmp = mm.mm_map_compare(ctx, m, m_ex)            # the paper's map statistics (Sect. 3.1)
    mm.mm_release_map(ctx, m)
    mm.mm_release_map(ctx, m_ex)
    t = min(times)
    out["fig1"] = {"ms": t, "equivalent_interactions_per_s": st["interactions"] / (t * 1e-3),
                   "speedup_vs_exact": exact_ms / t, "far_bound_re": st["far_bound"],
                   "rays_moved_vs_exact_fraction": float(np.abs(far.astype(np.int64) - ex).sum()) / 2 / st["rays_shot"],
                   "vs_exact_rms_delta_m": cmp["rms_dm"], "vs_exact_ks_probability": cmp["ks_p"],
                   "far_block_used": st["far_block"]}
    f2 = synth.lens_field(25000, 250.0, 3)
    lh2 = mm.mm_create_lenses_from(ctx, f2.x, f2.y, f2.m)
    cfg2 = dict(sigma=0.8, gamma=0.3, smooth_frac=0.5, side=40.0, npix_side=2048, nrays=500.0)
    times = []
    for _ in range(2):
        m = mm.mm_shoot(ctx, lh2, mm.params(**cfg2, precision=mm.MM_FAR32))
        times.append(mm.mm_last_kernel_ms(ctx)[0])
        _, st2 = mm.mm_map_fetch(ctx, m, want_counts=False)
        mm.mm_release_map(ctx, m)
    mm.mm_release_lenses(ctx, lh2)
    t2 = min(times)
    exact_rate = st_ex["interactions"] / (exact_ms * 1e-3)
    out["sigma08_nstar25000"] = {"ms": t2, "rays": st2["rays_shot"],
                                 "equivalent_interactions_per_s": st2["interactions"] / (t2 * 1e-3),
                                 "exact_estimated_s": st2["interactions"] / exact_rate,
                                 "far_bound_re": st2["far_bound"], "far_block_used": st2["far_block"]}
    return out


def kernel_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1005_5198_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def kernel_traffic():
    """DRAM bytes per launch of the shoot kernel from the committed ncu record, if it was taken
    on the current kernel source; otherwise None."""
    p = os.path.join(ROOT, "profiles", "shoot_fp32_traffic.json")
    try:
        rec = json.load(open(p))
        if rec.get("kernel_sha256") == kernel_sha256():
            return rec["dram_bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        pass
    return None


def reduce_over_ranks(dist, device, t_total, inter):
    """Whole-job figures: max time over ranks, sum of interactions over ranks."""
    if dist is None:
        return t_total, inter
    import torch
    tt = torch.tensor([t_total], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ti = torch.tensor([float(inter)], device=device, dtype=torch.float64)
    dist.all_reduce(ti)
    return float(tt.item()), float(ti.item())


def host_cpu():
    """The host CPU's model name and architecture (from lscpu, else /proc/cpuinfo, else platform)."""
    import platform
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return f"{model or platform.processor() or 'unknown'} ({platform.machine()}, {os.cpu_count()} logical CPUs)"


def cpu_baseline(seconds_target: float = 15.0):
    """The FP64 CPU oracle on a strided sample of the Fig. 1 map, host cores."""
    import oracle
    import synth
    from oracle import field
    n, r = field.nstar_rule(0.4, 0.0, 0.0, 20.0)
    f = synth.lens_field(n, r, SEED)
    cfg = dict(CFG1, margin=1.5)
    oracle.build()
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    _, tot = oracle.shoot_map(cfg, f, stride=CPU_STRIDE, threads=threads)
    dt = time.perf_counter() - t0
    inter = tot["shot"] * n
    return {"value": inter / dt, "unit": "interactions/s", "cores": threads, "kind": "oracle", "host": host_cpu(),
            "sample": f"Fig. 1 map, every {CPU_STRIDE}th ray row and column ({tot['shot']} rays x {n} lenses "
                      f"= {inter:.3e} interactions) in {dt:.1f} s, FP64, OpenMP"}


def profile_case(kind="fp32", window=4096):
    """Small case of the same kernel for ncu: a window x window-ray window at the centre of
    the Fig. 1 map (4096: 1.68e7 rays, 9.36e9 interactions), launched three times; kind
    "far" shoots it with the far-field approximation (MM_FAR32, default order, ratio and
    block; from 16384, 2048 blocks of 8 x 8 tiles, its work items are whole blocks as on
    the full map), kind "random" exactly with random rays (the window moved onto the tile grid)."""
    import paper_1005_5198_gb300 as mm
    import synth
    mm.build()
    ctx = mm.mm_init(0)
    n, r = lens_rule(mm, mm.params(**CFG1))
    f = synth.lens_field(n, r, SEED)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    g = mm.mm_geometry_of(mm.params(**CFG1))
    c = g["nx"] // 2
    h = window // 2
    i0, j0 = c - h, c - h
    extra = {}
    if kind == "random":                                 # random rays: a window on the 64 x 32 tile grid
        i0, j0 = i0 // 64 * 64, j0 // 32 * 32
        extra = dict(ray_mode=mm.MM_RAYS_RANDOM, ray_seed=SEED)
    p = mm.params(**CFG1, ray_rect=(i0, i0 + window, j0, j0 + window),
                  precision=mm.MM_FAR32 if kind == "far" else mm.MM_FP32C, **extra)
    for _ in range(3):
        m = mm.mm_shoot(ctx, lh, p)
        ms, _ = mm.mm_last_kernel_ms(ctx)
        _, st = mm.mm_map_fetch(ctx, m, want_counts=False)
        mm.mm_release_map(ctx, m)
        print(f"window {st['rays_shot']} rays: {ms:.3f} ms, {st['interactions'] / (ms * 1e-3):.3e} interactions/s")
    mm.mm_destroy(ctx)
    return 0


def far_scaling(counts=(10 ** 4, 10 ** 5, 10 ** 6, 10 ** 7, 10 ** 8)):
    """The far field (MM_FAR32, default order and ratio, automatic block) on the Fig. 1 geometry
    (sigma = 0.4, 1024^2 pixels of 20 R_E, 1.31e10 rays) with N* lenses spread over the disc that
    Eq. nstar gives for sigma_* = 0.4; one JSON line per N*. Lenses come from the library's seeded
    generator; the time is block preparation + shoot (CUDA events), the best of two; first_ms is the
    first map, which for grouped maps also builds the lens tree."""
    import paper_1005_5198_gb300 as mm
    mm.build()
    ctx = mm.mm_init(0)
    try:
        for n in counts:
            p = mm.params(**CFG1, nstar=n, precision=mm.MM_FAR32)
            lh = mm.mm_create_lenses(ctx, p)
            times, st = [], None
            for _ in range(2):
                m = mm.mm_shoot(ctx, lh, p)
                times.append(mm.mm_last_kernel_ms(ctx)[0])
                _, st = mm.mm_map_fetch(ctx, m, want_counts=False)
                mm.mm_release_map(ctx, m)
            best = min(times)
            mm.mm_release_lenses(ctx, lh)
            print(json.dumps({"nstar": n, "ms": best, "first_ms": times[0], "rays": st["rays_shot"],
                              "far_block": st["far_block"], "far_group": st["far_group"],
                              "far_bound_re": st["far_bound"], "mu_mean": st["mu_mean"],
                              "exact_interactions": st["interactions"],
                              "equivalent_interactions_per_s": st["interactions"] / (best * 1e-3)}), flush=True)
    finally:
        mm.mm_destroy(ctx)
    return 0


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import synth
    from oracle import field
    n, r = field.nstar_rule(0.4, 0.0, 0.0, 20.0)
    f = synth.lens_field(n, r, SEED)
    cfg = dict(CFG1, margin=1.5)
    oracle.build()
    threads = oracle.max_threads()
    stride = 24                                     # 1/576 of the map per step
    for _ in range(args.warmup):
        oracle.shoot_map(cfg, f, stride=stride, threads=threads)
    times, shot = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, tot = oracle.shoot_map(cfg, f, stride=stride, threads=threads)
        times.append(time.perf_counter() - t0)
        shot = tot["shot"]
    inter = shot * n
    value = inter * len(times) / sum(times)
    line = {"metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": f"every {stride}th ray row and column per step"},
            "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": threads, "kind": "oracle",
                             "host": host_cpu(),
                             "sample": f"every {stride}th ray row and column of the Fig. 1 map per step "
                                       f"({shot} rays x {n} lenses)"},
            "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the far-field, batch and serving phases")
    ap.add_argument("--wave-ms", type=float, default=12.0, help="serving: target device time of one wave")
    ap.add_argument("--serve-priority", type=float, default=0.8,
                    help="serving: share of each wave given shortest remaining work first (0: processor sharing)")
    ap.add_argument("--profile-window", type=int, default=4096, help="--profile-case: window side in rays")
    ap.add_argument("--clocks-dir", default=None,
                    help="where the nvidia-smi samples of the timed region go (clocks_rank<N>.csv; default: the "
                         "system's temporary directory)")
    ap.add_argument("--profile-case", nargs="?", const="fp32", choices=["fp32", "far", "random", "downstream"],
                    help="for ncu captures, then exit: shoot a window (--profile-window, 4096^2 rays) of the Fig. 1 map "
                         "three times, exactly (fp32), with the far-field approximation MM_FAR32 (far) or exactly with "
                         "random rays (random); or run the map statistics and light curves on two 8192^2 maps "
                         "(downstream)")
    ap.add_argument("--far-scaling", action="store_true",
                    help="time the far field on the Fig. 1 geometry for N* = 1e4 .. 1e8 and exit")
    ap.add_argument("--alu-rates", action="store_true",
                    help="build and run the arithmetic-pipe probe (FFMA, FFMA2, MUFU, DFMA and the shooting "
                         "mix per SM per clock: the roofline's denominators) and exit")
    args = ap.parse_args()
    if args.alu_rates:
        from paper_1005_5198_gb300.buildlib import build_alu_rates
        return subprocess.run([build_alu_rates()]).returncode
    if args.far_scaling:
        return far_scaling()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case == "downstream":               # map statistics and light curves (ncu captures)
        import paper_1005_5198_gb300 as mm
        mm.build()
        ctx = mm.mm_init(0)
        print(json.dumps(downstream_phase(mm, ctx, fma_peak_per_s=lane_peak_per_s(device_sms(0)))))
        mm.mm_destroy(ctx)
        return 0
    if args.profile_case:
        return profile_case(args.profile_case, args.profile_window)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    import torch
    import paper_1005_5198_gb300 as mm
    import synth

    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    mm.build()
    ctx = mm.mm_init(local, 0, stream.cuda_stream)
    sms = device_sms(local)
    peak = fp32_peak_tflops(sms)

    n, r = lens_rule(mm, mm.params(**CFG1))
    f = synth.lens_field(n, r, SEED + rank)
    lh = mm.mm_create_lenses_from(ctx, f.x, f.y, f.m)
    p = mm.params(**CFG1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")   # > 129 MB L2

    def step():
        m = mm.mm_shoot(ctx, lh, p)
        kms, launches = mm.mm_last_kernel_ms(ctx)
        _, st = mm.mm_map_fetch(ctx, m, want_counts=False)
        mm.mm_release_map(ctx, m)
        return st, kms, launches

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    step_ms, kern_ms, launches, inter = [], [], 0, 0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local, args.clocks_dir) as clk:
        for k in range(args.steps):
            flush.fill_(k & 0xFF)                       # evict L2 between timed steps (outside the events)
            ev[k][0].record(stream)
            st, kms, nl = step()
            ev[k][1].record(stream)
            kern_ms.append(kms)
            launches += nl
            inter += st["interactions"]
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = sum(step_ms) * 1e-3
    t_total, inter = reduce_over_ranks(dist, f"cuda:{local}", t_total, inter)
    value = inter / t_total
    maps_per_s = world * args.steps / t_total

    # ---- e2e through the public API with host buffers (pinned) ----
    hx = torch.from_numpy(f.x).pin_memory().numpy()
    hy = torch.from_numpy(f.y).pin_memory().numpy()
    hm = torch.from_numpy(f.m).pin_memory().numpy()
    hc = torch.empty(CFG1["npix_side"] ** 2, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    e2e_times = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = mm.mm_create_lenses_from(ctx, hx, hy, hm)
        m = mm.mm_shoot(ctx, h, p)
        counts, st = mm.mm_map_fetch(ctx, m, counts=hc)
        mm.mm_release_map(ctx, m)
        mm.mm_release_lenses(ctx, h)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    e2e_value = st["interactions"] * len(e2e_times) / sum(e2e_times)
    h2d = 3 * f.x.nbytes
    d2h = hc.nbytes + 16

    # ---- plain FP64 kernel on a window of the same map ----
    g = mm.mm_geometry_of(p)
    c = g["nx"] // 2
    win = (c - 1024, c + 1024, c - 512, c + 512)
    m64 = mm.mm_shoot(ctx, lh, mm.params(**CFG1, precision=mm.MM_FP64, ray_rect=win))
    ms64, _ = mm.mm_last_kernel_ms(ctx)
    _, st64 = mm.mm_map_fetch(ctx, m64, want_counts=False)
    mm.mm_release_map(ctx, m64)
    fp64 = {"value": st64["interactions"] / (ms64 * 1e-3), "unit": "interactions/s",
            "sample": f"2048 x 1024-ray window at the grid centre ({st64['interactions']:.3e} interactions)"}

    # ---- batched persistent launch and served stream (scaled config-3 / config-4 shapes) ----
    extra = {}
    if not args.no_extras and world == 1:
        extra["config2_exact"] = config2_phase(mm, ctx, sms)
        extra["far_field"] = far_phase(mm, ctx, lh, sum(kern_ms) / len(kern_ms))
        extra["random_rays"] = random_phase(mm, ctx, lh, sum(kern_ms) / len(kern_ms), sms)
        extra["downstream"] = downstream_phase(mm, ctx, fma_peak_per_s=lane_peak_per_s(sms))
        extra["batch"] = config3_phase(mm, ctx, sms)
        extra["batch_scaled"] = scaled_batch_phase(mm, ctx, sms)
        extra["serving"] = config4_phase(mm, ctx, extra["batch"]["batched_interactions_per_s"], args)

    clocks = clk.summary()
    kmean = sum(kern_ms) / len(kern_ms)
    achieved = FLOP_PER_INTERACTION * (inter / (world * args.steps)) / (kmean * 1e-3) / 1e12
    traffic = kernel_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "FP32 compensated (MM_FP32C)",
                   "l2": "flushed between timed steps (256 MiB write outside the step events)",
                   "parallelism": f"{world} independent maps, one per GPU"},
        "maps_per_s": maps_per_s,
        "e2e": {"value": e2e_value, "unit": "interactions/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "what": "mm_create_lenses_from (pinned host) + mm_shoot + mm_map_fetch (pinned host) per step"},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"recipe unit counts: {sms} SMs (from the device) x 128 FP32 lanes x 2 FLOP "
                                    f"x 2070 MHz",
                     "kernel_ms": kmean,
                     "frac_at_measured_clock": (achieved / (peak * clocks["sm_mhz"] / SM_MAX_MHZ)
                                                if clocks.get("sm_mhz") else None),
                     # against the FFMA rate the pipe probe measured (125.1 of 128 lane operations per
                     # SM per clock) at the maximum clock
                     "frac_of_measured_ffma": achieved / fp32_peak_tflops(sms, FFMA_MEASURED_LANE_OPS),
                     "measured_ffma_lane_ops_per_sm_clk": FFMA_MEASURED_LANE_OPS,
                     # the irreducible FP32 lane operations of an interaction (2 subtractions,
                     # 1 multiply, 3 FMAs) per second, against the FP32 lane peak
                     "useful_frac": USEFUL_OPS_PER_INTERACTION * (inter / (world * args.steps)) / (kmean * 1e-3)
                                    / lane_peak_per_s(sms),
                     "useful_ops_per_interaction": USEFUL_OPS_PER_INTERACTION},
        "fp64": fp64,
        "fp32_over_fp64": value / world / fp64["value"],
        "clocks": clocks,
    }
    line.update(extra)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    mm.mm_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
