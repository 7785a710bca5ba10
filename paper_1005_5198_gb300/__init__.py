"""Python binding of libmm (GB300 direct inverse ray-shooting of microlensing maps).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels behind the C ABI of include/mm.h. The functions keep
the C names (mm_init, mm_create_lenses, mm_shoot, mm_map_fetch, mm_submit,
mm_poll, ...) and raise MMError on a negative status. The library must have
been built (`build()`); importing this package without it raises, there is
no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

from .buildlib import CHECKED_LIB, LIB, up_to_date  # noqa: F401
from .buildlib import build as _build_lib

_checked = False


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libmm.so (the checked variant after use_checked_build()) if it is out of date."""
    return _build_lib(force=force, verbose=verbose, checked=_checked)


def use_checked_build() -> None:
    """Load the checked build (every guarded device access tests its index; a failure is reported
    as MM_EDEVICE "bounds check failed"). Call before the first use of the library."""
    global LIB, _checked
    if _lib is not None:
        raise RuntimeError("the library is already loaded")
    _checked = True
    LIB = _build_lib(checked=True)

MM_OK, MM_EINVAL, MM_ENOMEM, MM_EBUSY, MM_ENOTFOUND = 0, -1, -2, -3, -4
MM_ETIMEDOUT, MM_EDEVICE, MM_EAGAIN, MM_ECANCELED = -5, -6, -7, -8
MM_FP32C, MM_FP64, MM_FAR32 = 0, 1, 2
MM_MASS_UNIT, MM_MASS_LOGNORMAL = 0, 1
MM_RAYS_LATTICE, MM_RAYS_RANDOM = 0, 1
MM_PROFILE_GAUSSIAN, MM_PROFILE_DISC = 0, 1
MM_MAP_MU, MM_MAP_DELTA_M = 0, 1
MM_INJECT_NONE, MM_INJECT_COMPARE_NO_COPY, MM_INJECT_DISC_NO_COPY = 0, 1, 2


class MMError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


class mm_params(C.Structure):
    _fields_ = [("sigma", C.c_double), ("gamma", C.c_double), ("smooth_frac", C.c_double), ("side_re", C.c_double),
                ("npix_side", C.c_int32), ("nrays_per_pix", C.c_double), ("shoot_margin", C.c_double),
                ("precision", C.c_int32), ("nstar", C.c_int64), ("disc_radius", C.c_double),
                ("mass_model", C.c_int32), ("mass_mu", C.c_double), ("mass_s", C.c_double), ("seed", C.c_uint64),
                ("ray_rect", C.c_int64 * 4), ("far_order", C.c_int32), ("far_ratio", C.c_double),
                ("far_block", C.c_int32), ("far_group_order", C.c_int32), ("far_group_theta", C.c_double),
                ("far_group_leaf", C.c_int32), ("ray_mode", C.c_int32), ("ray_seed", C.c_uint64)]


class mm_stats(C.Structure):
    _fields_ = [("rays_shot", C.c_uint64), ("rays_in", C.c_uint64), ("rays_out", C.c_uint64),
                ("interactions", C.c_uint64), ("nx", C.c_uint64), ("ny", C.c_uint64), ("nstar", C.c_int64),
                ("seconds", C.c_double), ("mu_mean", C.c_double), ("lens_splits", C.c_int32),
                ("far_bound", C.c_double), ("far_block", C.c_int32), ("far_group", C.c_int32)]


class mm_compare(C.Structure):
    _fields_ = [("rms_dm", C.c_double), ("n_rms", C.c_int64), ("zero_a", C.c_int64), ("zero_b", C.c_int64),
                ("ks_d", C.c_double), ("ks_p", C.c_double), ("mean_mu_a", C.c_double), ("mean_mu_b", C.c_double)]


class mm_serve_stats_t(C.Structure):
    _fields_ = [("waves", C.c_uint64), ("items", C.c_uint64), ("interactions", C.c_double),
                ("completed", C.c_uint64), ("cancelled", C.c_uint64), ("failed", C.c_uint64),
                ("queued", C.c_int32), ("preparing", C.c_int32), ("active", C.c_int32)]


class mm_geometry(C.Structure):
    _fields_ = [("pix", C.c_double), ("delta", C.c_double), ("width", C.c_double), ("height", C.c_double),
                ("nx", C.c_int64), ("ny", C.c_int64), ("nstar", C.c_int64), ("disc_radius", C.c_double),
                ("mu_theory", C.c_double), ("far_block", C.c_int32), ("far_group", C.c_int32)]


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"libmm.so is not built ({LIB}); run paper_1005_5198_gb300.build() first")
    lib = C.CDLL(LIB)
    P, U64, I64, D = C.POINTER, C.c_uint64, C.c_int64, C.c_double
    sig = {
        "mm_init": [P(C.c_void_p), C.c_int, C.c_size_t, C.c_void_p],
        "mm_destroy": [C.c_void_p],
        "mm_params_default": [P(mm_params)],
        "mm_geometry_of": [P(mm_params), P(mm_geometry)],
        "mm_create_lenses": [C.c_void_p, P(mm_params), P(U64)],
        "mm_create_lenses_from": [C.c_void_p, P(D), P(D), P(D), I64, P(U64)],
        "mm_lenses_fetch": [C.c_void_p, U64, P(D), P(D), P(D), I64],
        "mm_lenses_count": [C.c_void_p, U64, P(I64)],
        "mm_release_lenses": [C.c_void_p, U64],
        "mm_shoot": [C.c_void_p, U64, P(mm_params), P(U64)],
        "mm_shoot_batch": [C.c_void_p, C.c_int32, P(U64), P(mm_params), P(U64)],
        "mm_shoot_into": [C.c_void_p, U64, P(mm_params), U64],
        "mm_map_restore": [C.c_void_p, U64, P(mm_params), P(C.c_uint32), C.c_size_t, P(mm_stats), P(U64)],
        "mm_map_fetch": [C.c_void_p, U64, P(C.c_uint32), C.c_size_t, P(mm_stats)],
        "mm_map_device_ptr": [C.c_void_p, U64, P(C.c_void_p), P(C.c_size_t)],
        "mm_map_fetch_mu": [C.c_void_p, U64, C.c_int32, P(C.c_float), C.c_size_t, P(I64)],
        "mm_release_map": [C.c_void_p, U64],
        "mm_submit": [C.c_void_p, U64, P(mm_params), P(U64)],
        "mm_poll": [C.c_void_p, U64, P(C.c_int), P(U64)],
        "mm_wait": [C.c_void_p, U64, I64, P(U64)],
        "mm_cancel": [C.c_void_p, U64],
        "mm_req_times": [C.c_void_p, U64, P(D), P(D)],
        "mm_serve_stats": [C.c_void_p, P(mm_serve_stats_t)],
        "mm_serve_config": [C.c_void_p, C.c_int32, C.c_int32, D],
        "mm_serve_priority": [C.c_void_p, D],
        "mm_serve_plan": [P(C.c_uint64), P(D), C.c_int32, D, D, C.c_uint64, P(C.c_uint64)],
        "mm_autotune": [C.c_void_p, P(mm_params), P(C.c_int32)],
        "mm_set_variant": [C.c_void_p, C.c_int32],
        "mm_variant_count": [],
        "mm_variant_name": [C.c_int32],
        "mm_set_layout": [C.c_void_p, C.c_int32],
        "mm_get_layout": [C.c_void_p, P(C.c_int32)],
        "mm_layout_count": [],
        "mm_layout_name": [C.c_int32],
        "mm_debug_deflect": [C.c_void_p, U64, P(mm_params), P(I64), P(I64), I64, P(D), P(I64)],
        "mm_debug_inject": [C.c_void_p, C.c_int32],
        "mm_last_kernel_ms": [C.c_void_p, P(D), P(C.c_int32)],
        "mm_shoot_noalloc": [C.c_void_p, C.c_void_p, C.c_void_p, I64, P(mm_params), C.c_void_p, C.c_void_p,
                             C.c_void_p],
        "mm_map_compare": [C.c_void_p, U64, U64, P(mm_compare)],
        "mm_map_convolve": [C.c_void_p, U64, C.c_int32, D, P(C.c_float), C.c_size_t],
        "mm_map_lightcurve": [C.c_void_p, U64, C.c_int32, D, D, D, D, D, I64, P(D)],
        "mm_strerror": [C.c_int],
        "mm_last_error": [],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.mm_variant_name.restype = C.c_char_p
    lib.mm_layout_name.restype = C.c_char_p
    lib.mm_strerror.restype = C.c_char_p
    lib.mm_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def lib():
    return _load()


def _check(rc: int, where: str):
    if rc < 0:
        raise MMError(rc, where, (_load().mm_last_error() or b"").decode())
    return rc


def params(**kw) -> mm_params:
    """mm_params with the library defaults (mm_params_default), overridden by keywords.
    `nrays` and `side` are accepted for nrays_per_pix and side_re; ray_rect takes a 4-tuple."""
    p = mm_params()
    _check(_load().mm_params_default(C.byref(p)), "mm_params_default")
    alias = {"nrays": "nrays_per_pix", "side": "side_re", "margin": "shoot_margin"}
    for k, v in kw.items():
        k = alias.get(k, k)
        if k == "ray_rect":
            p.ray_rect[:] = [int(t) for t in (v if v is not None else (-1, -1, -1, -1))]
        else:
            setattr(p, k, v)
    return p


def mm_geometry_of(p: mm_params) -> dict:
    g = mm_geometry()
    _check(_load().mm_geometry_of(C.byref(p), C.byref(g)), "mm_geometry_of")
    return {k: getattr(g, k) for k, _ in mm_geometry._fields_}


@dataclass
class Ctx:
    handle: C.c_void_p
    device: int
    released: bool = field(default=False)


def mm_init(device: int = 0, hbm_budget_bytes: int = 0, cuda_stream: int | None = None) -> Ctx:
    h = C.c_void_p()
    _check(_load().mm_init(C.byref(h), device, hbm_budget_bytes, C.c_void_p(cuda_stream or 0)), "mm_init")
    return Ctx(h, device)


def mm_destroy(ctx: Ctx) -> None:
    if not ctx.released:
        _check(_load().mm_destroy(ctx.handle), "mm_destroy")
        ctx.released = True


def mm_create_lenses(ctx: Ctx, p: mm_params) -> int:
    h = C.c_uint64()
    _check(_load().mm_create_lenses(ctx.handle, C.byref(p), C.byref(h)), "mm_create_lenses")
    return h.value


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def mm_create_lenses_from(ctx: Ctx, x, y, m) -> int:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    if not (x.shape == y.shape == m.shape) or x.ndim != 1:
        raise ValueError("x, y, m must be 1-D arrays of one length")
    h = C.c_uint64()
    _check(_load().mm_create_lenses_from(ctx.handle, _dptr(x), _dptr(y), _dptr(m), x.size, C.byref(h)),
           "mm_create_lenses_from")
    return h.value


def mm_lenses_count(ctx: Ctx, h: int) -> int:
    n = C.c_int64()
    _check(_load().mm_lenses_count(ctx.handle, h, C.byref(n)), "mm_lenses_count")
    return n.value


def mm_lenses_fetch(ctx: Ctx, h: int):
    n = mm_lenses_count(ctx, h)
    x, y, m = (np.zeros(n) for _ in range(3))
    _check(_load().mm_lenses_fetch(ctx.handle, h, _dptr(x), _dptr(y), _dptr(m), n), "mm_lenses_fetch")
    return x, y, m


def mm_release_lenses(ctx: Ctx, h: int) -> None:
    _check(_load().mm_release_lenses(ctx.handle, h), "mm_release_lenses")


def mm_shoot(ctx: Ctx, lenses: int, p: mm_params) -> int:
    h = C.c_uint64()
    _check(_load().mm_shoot(ctx.handle, lenses, C.byref(p), C.byref(h)), "mm_shoot")
    return h.value


def mm_shoot_batch(ctx: Ctx, lenses, plist) -> list[int]:
    n = len(plist)
    parr = (mm_params * n)(*plist)
    larr = (C.c_uint64 * n)(*(lenses if lenses is not None else [0] * n))
    out = (C.c_uint64 * n)()
    _check(_load().mm_shoot_batch(ctx.handle, n, larr, parr, out), "mm_shoot_batch")
    return list(out)


def mm_shoot_into(ctx: Ctx, lenses: int, p: mm_params, m: int) -> None:
    """Add the rays of p.ray_rect to an existing map (shooting in parts / resuming)."""
    _check(_load().mm_shoot_into(ctx.handle, lenses, C.byref(p), m), "mm_shoot_into")


def _stats_dict(st: mm_stats) -> dict:
    return {k: getattr(st, k) for k, _ in mm_stats._fields_}


def mm_map_restore(ctx: Ctx, lenses: int, p: mm_params, counts: np.ndarray, stats: dict) -> int:
    """A new map from a checkpoint (the counts and stats dict of mm_map_fetch; fields the dict lacks
    are 0)."""
    c = np.ascontiguousarray(counts, dtype=np.uint32).ravel()
    st = mm_stats(**{k: stats.get(k, 0) for k, _ in mm_stats._fields_})
    out = C.c_uint64()
    _check(_load().mm_map_restore(ctx.handle, lenses, C.byref(p), c.ctypes.data_as(C.POINTER(C.c_uint32)), c.size,
                                  C.byref(st), C.byref(out)), "mm_map_restore")
    return out.value


def mm_map_fetch(ctx: Ctx, m: int, counts: np.ndarray | None = None, want_counts: bool = True):
    """(uint32 counts [N_side, N_side] or None, stats dict). `counts` may be a preallocated
    (pinned or pageable) uint32 array of N_side^2 elements to fill."""
    st = mm_stats()
    if not want_counts:
        _check(_load().mm_map_fetch(ctx.handle, m, None, 0, C.byref(st)), "mm_map_fetch")
        return None, _stats_dict(st)
    ptr, n = C.c_void_p(), C.c_size_t()
    _check(_load().mm_map_device_ptr(ctx.handle, m, C.byref(ptr), C.byref(n)), "mm_map_device_ptr")
    if counts is None:
        counts = np.zeros(n.value, dtype=np.uint32)
    if counts.dtype != np.uint32 or counts.size != n.value or not counts.flags.c_contiguous:
        raise ValueError("counts must be a contiguous uint32 array of N_side^2 elements")
    _check(_load().mm_map_fetch(ctx.handle, m, counts.ctypes.data_as(C.POINTER(C.c_uint32)), n.value,
                                C.byref(st)), "mm_map_fetch")
    side = int(round(n.value ** 0.5))
    return counts.reshape(side, side), _stats_dict(st)


def mm_map_fetch_mu(ctx: Ctx, m: int, kind: int = MM_MAP_MU):
    """(float32 [N_side, N_side] of mu = N / N_rays, or of Delta m with empty pixels clamped to one
    ray (kind MM_MAP_DELTA_M), computed on the device; number of empty pixels)."""
    _, n = mm_map_device_ptr(ctx, m)
    out = np.zeros(n, dtype=np.float32)
    empty = C.c_int64()
    _check(_load().mm_map_fetch_mu(ctx.handle, m, kind, out.ctypes.data_as(C.POINTER(C.c_float)), n,
                                   C.byref(empty)), "mm_map_fetch_mu")
    side = int(round(n ** 0.5))
    return out.reshape(side, side), empty.value


def mm_map_device_ptr(ctx: Ctx, m: int) -> tuple[int, int]:
    ptr, n = C.c_void_p(), C.c_size_t()
    _check(_load().mm_map_device_ptr(ctx.handle, m, C.byref(ptr), C.byref(n)), "mm_map_device_ptr")
    return ptr.value, n.value


def mm_release_map(ctx: Ctx, m: int) -> None:
    _check(_load().mm_release_map(ctx.handle, m), "mm_release_map")


def mm_submit(ctx: Ctx, lenses: int, p: mm_params) -> int:
    h = C.c_uint64()
    _check(_load().mm_submit(ctx.handle, lenses, C.byref(p), C.byref(h)), "mm_submit")
    return h.value


def mm_poll(ctx: Ctx, req: int):
    """(done, map handle or None)."""
    done, m = C.c_int(), C.c_uint64()
    _check(_load().mm_poll(ctx.handle, req, C.byref(done), C.byref(m)), "mm_poll")
    return bool(done.value), (m.value if done.value else None)


def mm_wait(ctx: Ctx, req: int, timeout_s: float | None = None) -> int:
    m = C.c_uint64()
    t = -1 if timeout_s is None else int(timeout_s * 1e9)
    _check(_load().mm_wait(ctx.handle, req, t, C.byref(m)), "mm_wait")
    return m.value


def mm_cancel(ctx: Ctx, req: int) -> None:
    _check(_load().mm_cancel(ctx.handle, req), "mm_cancel")


def mm_req_times(ctx: Ctx, req: int) -> tuple[float, float]:
    q, t = C.c_double(), C.c_double()
    _check(_load().mm_req_times(ctx.handle, req, C.byref(q), C.byref(t)), "mm_req_times")
    return q.value, t.value


def mm_serve_stats(ctx: Ctx) -> dict:
    """Serving counters: waves, items, interactions shot, requests completed / cancelled / failed,
    and the requests queued, being prepared and active now."""
    out = mm_serve_stats_t()
    _check(_load().mm_serve_stats(ctx.handle, C.byref(out)), "mm_serve_stats")
    return {k: getattr(out, k) for k, _ in mm_serve_stats_t._fields_}


def mm_serve_config(ctx: Ctx, max_active: int = 0, max_queued: int = 0, wave_ms: float = 0.0) -> None:
    _check(_load().mm_serve_config(ctx.handle, max_active, max_queued, wave_ms), "mm_serve_config")


def mm_serve_priority(ctx: Ctx, priority_share: float) -> None:
    _check(_load().mm_serve_priority(ctx.handle, priority_share), "mm_serve_priority")


def mm_serve_plan(left, cost, budget: float, priority_share: float, min_items: int = 0) -> np.ndarray:
    """Items per map of one serving wave (host only, no GPU): see mm_serve_plan in mm.h."""
    left = np.ascontiguousarray(left, dtype=np.uint64)
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    if left.shape != cost.shape or left.ndim != 1:
        raise ValueError("left and cost must be 1-D arrays of the same length")
    take = np.zeros_like(left)
    u64p, f64p = C.POINTER(C.c_uint64), C.POINTER(C.c_double)
    _check(_load().mm_serve_plan(left.ctypes.data_as(u64p), cost.ctypes.data_as(f64p), len(left), budget,
                                 priority_share, min_items, take.ctypes.data_as(u64p)), "mm_serve_plan")
    return take


def mm_autotune(ctx: Ctx, p: mm_params) -> int:
    v = C.c_int32()
    _check(_load().mm_autotune(ctx.handle, C.byref(p), C.byref(v)), "mm_autotune")
    return v.value


def mm_set_variant(ctx: Ctx, variant: int) -> None:
    _check(_load().mm_set_variant(ctx.handle, variant), "mm_set_variant")


def mm_variant_count() -> int:
    return _load().mm_variant_count()


def mm_variant_name(v: int) -> str:
    return _load().mm_variant_name(v).decode()


def mm_set_layout(ctx: Ctx, layout: int) -> None:
    _check(_load().mm_set_layout(ctx.handle, layout), "mm_set_layout")


def mm_get_layout(ctx: Ctx) -> int:
    v = C.c_int32()
    _check(_load().mm_get_layout(ctx.handle, C.byref(v)), "mm_get_layout")
    return v.value


def mm_layout_count() -> int:
    return _load().mm_layout_count()


def mm_layout_name(v: int) -> str:
    return _load().mm_layout_name(v).decode()


def mm_debug_inject(ctx: Ctx, kind: int) -> None:
    """Arm a one-shot device-side failure for the next call of the named kind (test hook)."""
    _check(_load().mm_debug_inject(ctx.handle, kind), "mm_debug_inject")


def mm_debug_deflect(ctx: Ctx, lenses: int, p: mm_params, ray_i, ray_j):
    """(alpha [n, 2] float64, pixel [n] int64, -1 = out) through the map kernel's code."""
    ri = np.ascontiguousarray(ray_i, dtype=np.int64)
    rj = np.ascontiguousarray(ray_j, dtype=np.int64)
    n = ri.size
    alpha = np.zeros((n, 2), dtype=np.float64)
    pix = np.zeros(n, dtype=np.int64)
    I64P = C.POINTER(C.c_int64)
    _check(_load().mm_debug_deflect(ctx.handle, lenses, C.byref(p), ri.ctypes.data_as(I64P), rj.ctypes.data_as(I64P),
                                    n, _dptr(alpha), pix.ctypes.data_as(I64P)), "mm_debug_deflect")
    return alpha, pix


def mm_last_kernel_ms(ctx: Ctx) -> tuple[float, int]:
    ms, n = C.c_double(), C.c_int32()
    _check(_load().mm_last_kernel_ms(ctx.handle, C.byref(ms), C.byref(n)), "mm_last_kernel_ms")
    return ms.value, n.value


def mm_shoot_noalloc(x_ptr: int, y_ptr: int, m_ptr: int, nstar: int, p: mm_params, counts_ptr: int,
                     totals_ptr: int, cuda_stream: int = 0) -> None:
    """One FP32 map into caller-owned device buffers without any allocation by the library
    (see include/mm.h). All pointers are device addresses (ints) on the current device."""
    _check(_load().mm_shoot_noalloc(C.c_void_p(x_ptr), C.c_void_p(y_ptr), C.c_void_p(m_ptr or None), nstar,
                                    C.byref(p), C.c_void_p(counts_ptr), C.c_void_p(totals_ptr),
                                    C.c_void_p(cuda_stream or None)), "mm_shoot_noalloc")


def mm_map_compare(ctx: Ctx, a: int, b: int) -> dict:
    """RMS difference of Delta m and the K-S test between two maps (Sect. 3.1), on the device."""
    out = mm_compare()
    _check(_load().mm_map_compare(ctx.handle, a, b, C.byref(out)), "mm_map_compare")
    return {k: getattr(out, k) for k, _ in mm_compare._fields_}


def mm_map_convolve(ctx: Ctx, m: int, profile: int, size_re: float) -> np.ndarray:
    """Magnification map of an extended source (float32 [N_side, N_side], NaN near the edges)."""
    _, n = mm_map_device_ptr(ctx, m)
    out = np.zeros(n, dtype=np.float32)
    _check(_load().mm_map_convolve(ctx.handle, m, profile, size_re, out.ctypes.data_as(C.POINTER(C.c_float)), n),
           "mm_map_convolve")
    side = int(round(n ** 0.5))
    return out.reshape(side, side)


def mm_map_lightcurve(ctx: Ctx, m: int, profile: int, size_re: float, start, end, n_points: int) -> np.ndarray:
    """Magnification along a straight source track from start=(y1, y2) to end (Einstein radii)."""
    out = np.zeros(n_points, dtype=np.float64)
    _check(_load().mm_map_lightcurve(ctx.handle, m, profile, size_re, start[0], start[1], end[0], end[1],
                                     n_points, _dptr(out)), "mm_map_lightcurve")
    return out


def mm_strerror(code: int) -> str:
    return _load().mm_strerror(code).decode()


EXPORTED = [
    "mm_init", "mm_destroy", "mm_params_default", "mm_geometry_of", "mm_create_lenses", "mm_create_lenses_from",
    "mm_lenses_fetch", "mm_lenses_count", "mm_release_lenses", "mm_shoot", "mm_shoot_batch", "mm_shoot_into",
    "mm_map_restore", "mm_map_fetch", "mm_map_fetch_mu",
    "mm_map_device_ptr", "mm_release_map", "mm_submit", "mm_poll", "mm_wait", "mm_cancel", "mm_req_times", "mm_serve_stats",
    "mm_serve_config", "mm_serve_priority", "mm_serve_plan", "mm_autotune", "mm_set_variant", "mm_variant_count", "mm_variant_name", "mm_set_layout",
    "mm_get_layout", "mm_layout_count", "mm_layout_name", "mm_debug_deflect", "mm_debug_inject",
    "mm_last_kernel_ms", "mm_shoot_noalloc", "mm_map_compare", "mm_map_convolve",
    "mm_map_lightcurve", "mm_strerror", "mm_last_error",
]
