"""Lens-field rules of the oracle (TEST INFRASTRUCTURE; see the package docstring).

Eq. nstar: N* = sigma_* A / (pi <M>) with A = pi R^2 the area of the lens
disc, i.e. N* = sigma_* R^2 / <M> and R = sqrt(N* <M> / sigma_*).

Disc radius (Sect. 2, the paragraph after Eq. nstar): the paper puts the
lenses in a circle wider than the long axis of the mapped-back source region
but does not give the radius. Reading: R = (margin/2) sqrt((L/|a|)^2 +
(L/|b|)^2) + 2 R_E -- half the diagonal of the shot rectangle plus 2
Einstein radii. With margin 1.5 and L = 20 this reproduces 19 of the 20 N*
values printed in Sect. 3.1 (the sigma and gamma sweeps); the remaining one
(sigma = 0.9: 41267 here, 41257 printed) differs by 0.02 %.

Eq. mutheory: mu_av = 1 / ((1 - sigma)^2 - gamma^2).
"""
from __future__ import annotations

import math


def mean_mass(model: int, mu: float = 0.0, s: float = 0.5) -> float:
    """<M>: 1 for unit masses, exp(mu + s^2/2) for lognormal(mu, s)."""
    return 1.0 if model == 0 else math.exp(mu + 0.5 * s * s)


def mu_theory(sigma: float, gamma: float) -> float:
    """Mean magnification without microlensing (Eq. mutheory); negative = parity flip."""
    return 1.0 / ((1.0 - sigma) ** 2 - gamma ** 2)


def disc_radius_rule(sigma: float, gamma: float, side: float, margin: float = 1.5) -> float:
    a = abs(1.0 - sigma - gamma)
    b = abs(1.0 - sigma + gamma)
    return 0.5 * margin * math.hypot(side / a, side / b) + 2.0


def nstar_for_radius(sigma_star: float, radius: float, mmean: float = 1.0) -> int:
    """Eq. nstar with A = pi R^2, rounded to the nearest integer."""
    return int(math.floor(sigma_star * radius * radius / mmean + 0.5))


def radius_for_nstar(nstar: int, sigma_star: float, mmean: float = 1.0) -> float:
    """Eq. nstar solved for the disc radius."""
    if sigma_star <= 0.0:
        raise ValueError("sigma_* must be > 0 to size a lens disc")
    return math.sqrt(nstar * mmean / sigma_star)


def nstar_rule(sigma: float, gamma: float, smooth_frac: float, side: float,
               margin: float = 1.5, mmean: float = 1.0) -> tuple[int, float]:
    """(N*, R) for a map when neither is given: R by the disc reading, N* by Eq. nstar."""
    sigma_star = (1.0 - smooth_frac) * sigma
    radius = disc_radius_rule(sigma, gamma, side, margin)
    if sigma_star <= 0.0:
        return 0, radius
    return nstar_for_radius(sigma_star, radius, mmean), radius
