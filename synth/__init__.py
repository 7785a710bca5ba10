"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module holds no arithmetic of the ray-shooting method: it only draws
random numbers and shapes them into lens fields and request parameters.
Everything here is deterministic in the seed.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014). The k-th output (k = 1, 2, ...) of a
generator seeded with s is mix64(s + k * 0x9E3779B97F4A7C15 mod 2^64), where
mix64 is the published finaliser (shifts 30/27/31, multipliers
0xBF58476D1CE4E5B9 and 0x94D049BB133111EB). A uniform double in [0, 1) is
the top 53 bits times 2^-53. The library's own C++ lens-field generator
implements the same definition independently; a test compares the two.

Lens fields (the paper places its lenses uniformly in a circle of area A,
Sect. 2, the paragraph after Eq. nstar):
  * positions: rejection sampling from the square [-R, R)^2, candidate c
    taking outputs 2c+1 and 2c+2 of the position stream, x = R(2u1-1),
    y = R(2u2-1), kept iff x*x + y*y < R*R (strict). Only IEEE-exact
    operations and single roundings, so every implementation agrees bit
    for bit.
  * masses: unit (1.0), or lognormal exp(mu + s z) with z from the
    Box-Muller cosine branch on outputs 2i+1, 2i+2 of the mass stream,
    u1 -> 1 - u1 so that the logarithm never sees zero.
  * stream seeds: the position stream is seeded with output 1 of
    SplitMix64(seed), the mass stream with output 2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1

MASS_UNIT = 0
MASS_LOGNORMAL = 1


def mix64(z: int) -> int:
    """SplitMix64 finaliser on one 64-bit integer."""
    z &= _MASK
    z = ((z ^ (z >> 30)) * _M1) & _MASK
    z = ((z ^ (z >> 27)) * _M2) & _MASK
    return z ^ (z >> 31)


def splitmix64(seed: int, k: np.ndarray) -> np.ndarray:
    """Outputs number k (k >= 1, uint64 array) of SplitMix64 seeded with `seed`."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + k * np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, k: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from outputs k of SplitMix64(seed)."""
    z = splitmix64(seed, k)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def stream_seeds(seed: int) -> tuple[int, int]:
    """(position-stream seed, mass-stream seed) derived from a field seed."""
    s = seed & _MASK
    return mix64(s + GOLDEN_GAMMA), mix64(s + 2 * GOLDEN_GAMMA)


@dataclass
class LensField:
    x: np.ndarray  # float64 [n]
    y: np.ndarray  # float64 [n]
    m: np.ndarray  # float64 [n]

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def disc_positions(n: int, radius: float, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """n points uniform in the open disc of the given radius (rejection sampling)."""
    pos_seed, _ = stream_seeds(seed)
    xs, ys = [], []
    have = 0
    cand = 0
    while have < n:
        batch = max(64, int((n - have) * 1.35) + 64)
        c = np.arange(cand, cand + batch, dtype=np.uint64)
        u1 = uniform01(pos_seed, np.uint64(2) * c + np.uint64(1))
        u2 = uniform01(pos_seed, np.uint64(2) * c + np.uint64(2))
        x = radius * (2.0 * u1 - 1.0)
        y = radius * (2.0 * u2 - 1.0)
        keep = (x * x + y * y) < radius * radius
        xs.append(x[keep])
        ys.append(y[keep])
        have += int(keep.sum())
        cand += batch
    return np.concatenate(xs)[:n].copy(), np.concatenate(ys)[:n].copy()


def masses(n: int, seed: int, model: int = MASS_UNIT, mu: float = 0.0, s: float = 0.5) -> np.ndarray:
    if model == MASS_UNIT:
        return np.ones(n, dtype=np.float64)
    if model != MASS_LOGNORMAL:
        raise ValueError(f"unknown mass model {model}")
    _, mass_seed = stream_seeds(seed)
    i = np.arange(n, dtype=np.uint64)
    u1 = 1.0 - uniform01(mass_seed, np.uint64(2) * i + np.uint64(1))
    u2 = uniform01(mass_seed, np.uint64(2) * i + np.uint64(2))
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    return np.exp(mu + s * z)


def lens_field(n: int, radius: float, seed: int, model: int = MASS_UNIT,
               mu: float = 0.0, s: float = 0.5) -> LensField:
    """A seeded lens field: n lenses uniform in a disc, unit or lognormal masses."""
    if n < 0:
        raise ValueError("n must be >= 0")
    if n == 0:
        e = np.zeros(0, dtype=np.float64)
        return LensField(e, e.copy(), e.copy())
    x, y = disc_positions(n, radius, seed)
    return LensField(x, y, masses(n, seed, model, mu, s))


# ---------------------------------------------------------------------------
# Request / map parameter mixes (shapes of the batched and served workloads).
# Only random draws: the caller derives N*, geometry and everything else.
# ---------------------------------------------------------------------------

@dataclass
class MapDraw:
    sigma: float
    gamma: float
    smooth_frac: float
    side: float
    npix_side: int
    nrays: float
    mass_model: int
    mass_mu: float
    mass_s: float
    seed: int


def map_mix(count: int, seed: int, *, guard: float = 0.05,
            sides=(256, 512, 1024), nrays=(100.0, 300.0, 1000.0),
            sigma=(0.2, 1.5), gamma=(0.0, 0.6), smooth=(0.0, 0.9), side=(10.0, 40.0)) -> list[MapDraw]:
    """`count` map parameter draws: sigma, gamma, s, L uniform, N_side and N_rays from
    the given sets, lognormal(0, 0.5) masses. Draws with min(|1-sigma-gamma|,
    |1-sigma+gamma|) < guard are redrawn (an ill-posed or near-critical map)."""
    out: list[MapDraw] = []
    k = 1
    while len(out) < count:
        u = uniform01(seed, np.arange(k, k + 7, dtype=np.uint64))
        k += 7
        sg = sigma[0] + (sigma[1] - sigma[0]) * u[0]
        gm = gamma[0] + (gamma[1] - gamma[0]) * u[1]
        if min(abs(1 - sg - gm), abs(1 - sg + gm)) < guard:
            continue
        out.append(MapDraw(
            sigma=float(sg), gamma=float(gm),
            smooth_frac=float(smooth[0] + (smooth[1] - smooth[0]) * u[2]),
            side=float(side[0] + (side[1] - side[0]) * u[3]),
            npix_side=int(sides[min(int(u[4] * len(sides)), len(sides) - 1)]),
            nrays=float(nrays[min(int(u[5] * len(nrays)), len(nrays) - 1)]),
            mass_model=MASS_LOGNORMAL, mass_mu=0.0, mass_s=0.5,
            seed=int(splitmix64(seed ^ 0x5EED, np.array([len(out) + 1], dtype=np.uint64))[0])))
    return out


def poisson_arrivals(count: int, rate_hz: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process: exponential gaps from uniforms."""
    u = uniform01(seed, np.arange(1, count + 1, dtype=np.uint64))
    gaps = -np.log1p(-u) / rate_hz
    return np.cumsum(gaps)
