"""Plain FP64 CPU oracle for direct inverse ray-shooting (TEST INFRASTRUCTURE).

Only the tests, the smoke check and the bench's CPU-baseline leg may import
this package. The library never does, and the library's code shares nothing
with it: this is an independent statement of the method written from the
paper (Eq. sigma, Eq. square, Eq. nstar, Eq. mutheory and the inverse
ray-shooting estimator of Sect. 2), used to prove the CUDA path right.

The arithmetic lives in `mm_oracle.c` (plain C, FP64, lenses summed in
index order, OpenMP over ray rows); `field.py` holds the lens-field rules.
Parameters are passed as a mapping with keys sigma, gamma, smooth_frac, side,
npix_side, nrays and margin (default 1.5), and optionally ray_mode (RAYS_LATTICE,
the default, or RAYS_RANDOM) and ray_seed.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

from .field import disc_radius_rule, mean_mass, mu_theory, nstar_for_radius, radius_for_nstar, nstar_rule  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mm_oracle.c")
_HDR = os.path.join(_HERE, "mm_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmm_oracle.so")
_lock = threading.Lock()
_lib = None


class _Params(C.Structure):
    _fields_ = [("sigma", C.c_double), ("gamma", C.c_double), ("smooth_frac", C.c_double),
                ("side", C.c_double), ("npix_side", C.c_int32), ("nrays", C.c_double),
                ("margin", C.c_double), ("ray_mode", C.c_int32), ("ray_seed", C.c_uint64)]


RAYS_LATTICE, RAYS_RANDOM = 0, 1


class _Far(C.Structure):
    _fields_ = [("order", C.c_int32), ("ratio", C.c_double), ("block_tiles", C.c_int32),
                ("group_order", C.c_int32), ("group_theta", C.c_double), ("group_leaf", C.c_int32)]


class _Geom(C.Structure):
    _fields_ = [("pix", C.c_double), ("delta", C.c_double), ("width", C.c_double),
                ("height", C.c_double), ("nx", C.c_int64), ("ny", C.c_int64)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE FP64: no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=c11", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            d, i64, u32, u64 = C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)
            lib.orc_geometry.argtypes = [C.POINTER(_Params), C.POINTER(_Geom)]
            lib.orc_map.argtypes = [C.POINTER(_Params), d, d, d, C.c_int64, C.c_int64, C.c_int64, C.c_int64,
                                    C.c_int64, C.c_int64, u32, u64, C.c_int]
            lib.orc_rays.argtypes = [C.POINTER(_Params), d, d, d, C.c_int64, i64, i64, C.c_int64, d, d, i64, C.c_int]
            lib.orc_far_map.argtypes = [C.POINTER(_Params), C.POINTER(_Far), d, d, d, C.c_int64, C.c_int64,
                                        C.c_int64, C.c_int64, C.c_int64, u32, u64, d, C.c_int]
            lib.orc_far_rays.argtypes = [C.POINTER(_Params), C.POINTER(_Far), d, d, d, C.c_int64, C.c_int64,
                                         C.c_int64, i64, i64, C.c_int64, d, d, i64, d, C.c_int]
            lib.orc_max_threads.restype = C.c_int
            _lib = lib
    return _lib


def _params(p) -> _Params:
    g = p.get if isinstance(p, dict) else (lambda k, dflt=None: getattr(p, k, dflt))
    return _Params(float(g("sigma")), float(g("gamma")), float(g("smooth_frac", 0.0) or 0.0),
                   float(g("side")), int(g("npix_side")), float(g("nrays")), float(g("margin", 1.5) or 1.5),
                   int(g("ray_mode", RAYS_LATTICE) or RAYS_LATTICE), int(g("ray_seed", 0) or 0))


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None and a.size else None


def geometry(p) -> dict:
    """Shot-rectangle geometry: pix, delta, width, height, nx, ny (Eq. square + lattice reading)."""
    g = _Geom()
    if _load().orc_geometry(C.byref(_params(p)), C.byref(g)) != 0:
        raise ValueError("ill-posed map parameters")
    return dict(pix=g.pix, delta=g.delta, width=g.width, height=g.height, nx=g.nx, ny=g.ny)


def _lens_arrays(field):
    x = np.ascontiguousarray(field.x, dtype=np.float64)
    y = np.ascontiguousarray(field.y, dtype=np.float64)
    m = np.ascontiguousarray(field.m, dtype=np.float64)
    return x, y, m


def shoot_map(p, field, rect=None, stride: int = 1, threads: int = 0):
    """uint32 counts [N_side, N_side] (row J along y2) and totals {shot, in, out}.
    rect = (i0, i1, j0, j1) restricts to a sub-rectangle of the global ray grid."""
    x, y, m = _lens_arrays(field)
    n = int(p["npix_side"] if isinstance(p, dict) else p.npix_side)
    counts = np.zeros(n * n, dtype=np.uint32)
    totals = np.zeros(3, dtype=np.uint64)
    i0, i1, j0, j1 = rect if rect is not None else (-1, -1, -1, -1)
    rc = _load().orc_map(C.byref(_params(p)), _ptr(x, C.c_double), _ptr(y, C.c_double), _ptr(m, C.c_double),
                         x.size, i0, i1, j0, j1, int(stride), _ptr(counts, C.c_uint32), _ptr(totals, C.c_uint64),
                         int(threads))
    if rc != 0:
        raise ValueError("oracle map failed (bad parameters)")
    return counts.reshape(n, n), dict(shot=int(totals[0]), inside=int(totals[1]), out=int(totals[2]))


def shoot_rays(p, field, ray_i, ray_j, threads: int = 0):
    """Per-ray alpha [n,2], source position y [n,2] and flat pixel index [n] (-1 = out)."""
    x, y, m = _lens_arrays(field)
    ri = np.ascontiguousarray(ray_i, dtype=np.int64)
    rj = np.ascontiguousarray(ray_j, dtype=np.int64)
    n = ri.size
    alpha = np.zeros((n, 2), dtype=np.float64)
    ysrc = np.zeros((n, 2), dtype=np.float64)
    pix = np.zeros(n, dtype=np.int64)
    if n == 0:
        return alpha, ysrc, pix
    rc = _load().orc_rays(C.byref(_params(p)), _ptr(x, C.c_double), _ptr(y, C.c_double), _ptr(m, C.c_double),
                          x.size, _ptr(ri, C.c_int64), _ptr(rj, C.c_int64), n, _ptr(alpha, C.c_double),
                          _ptr(ysrc, C.c_double), _ptr(pix, C.c_int64), int(threads))
    if rc != 0:
        raise ValueError("oracle rays failed (bad parameters)")
    return alpha, ysrc, pix


def _far(far) -> _Far:
    """far = {order P, ratio q, block_tiles bt} and, for grouped far lenses, group_order K (0: none),
    group_theta and group_leaf."""
    return _Far(int(far["order"]), float(far["ratio"]), int(far["block_tiles"]), int(far.get("group_order", 0)),
                float(far.get("group_theta", 0.5)), int(far.get("group_leaf", 64)))


def far_map(p, field, far, rect=None, threads: int = 0):
    """Far-field approximation of the map (the tree code's idea on blocks of rays, Sect. 2.1,
    Eq. hierarchical): far = {order P, ratio q, block_tiles bt}, plus group_order K, group_theta and
    group_leaf to group distant lenses by cells of a lens tree. Returns counts [N_side, N_side],
    totals {shot, in, out} and the largest truncation bound of any block."""
    x, y, m = _lens_arrays(field)
    n = int(p["npix_side"] if isinstance(p, dict) else p.npix_side)
    counts = np.zeros(n * n, dtype=np.uint32)
    totals = np.zeros(3, dtype=np.uint64)
    bmax = C.c_double(0.0)
    i0, i1, j0, j1 = rect if rect is not None else (-1, -1, -1, -1)
    rc = _load().orc_far_map(C.byref(_params(p)), C.byref(_far(far)), _ptr(x, C.c_double), _ptr(y, C.c_double),
                             _ptr(m, C.c_double), x.size, i0, i1, j0, j1, _ptr(counts, C.c_uint32),
                             _ptr(totals, C.c_uint64), C.byref(bmax), int(threads))
    if rc != 0:
        raise ValueError("oracle far-field map failed (bad parameters)")
    return counts.reshape(n, n), dict(shot=int(totals[0]), inside=int(totals[1]), out=int(totals[2])), bmax.value


def far_rays(p, field, far, ray_i, ray_j, origin=(0, 0), threads: int = 0):
    """Per-ray far-field alpha [n,2], source position [n,2], flat pixel [n] (-1 = out) and
    truncation bound [n]; blocks are counted from the rectangle origin (i0, j0)."""
    x, y, m = _lens_arrays(field)
    ri = np.ascontiguousarray(ray_i, dtype=np.int64)
    rj = np.ascontiguousarray(ray_j, dtype=np.int64)
    n = ri.size
    alpha = np.zeros((n, 2), dtype=np.float64)
    ysrc = np.zeros((n, 2), dtype=np.float64)
    pix = np.zeros(n, dtype=np.int64)
    bound = np.zeros(n, dtype=np.float64)
    if n == 0:
        return alpha, ysrc, pix, bound
    rc = _load().orc_far_rays(C.byref(_params(p)), C.byref(_far(far)), _ptr(x, C.c_double), _ptr(y, C.c_double),
                              _ptr(m, C.c_double), x.size, int(origin[0]), int(origin[1]), _ptr(ri, C.c_int64),
                              _ptr(rj, C.c_int64), n, _ptr(alpha, C.c_double), _ptr(ysrc, C.c_double),
                              _ptr(pix, C.c_int64), _ptr(bound, C.c_double), int(threads))
    if rc != 0:
        raise ValueError("oracle far-field rays failed (bad parameters)")
    return alpha, ysrc, pix, bound


def max_threads() -> int:
    return int(_load().orc_max_threads())
