"""Extended-source magnification of the oracle (TEST INFRASTRUCTURE; see the package docstring).

Sect. 1: a finite source's magnification at each position is the point-source
map convolved with its brightness profile. Readings (the same as the library's, written
independently): mu = N / N_rays per pixel; the profile is discretised on the
pixel grid and normalised to unit sum -- Gaussian w(i, j) = g(i) g(j) with
g(k) = exp(-(k p)^2 / (2 s^2)) for |k| <= ceil(4 s / p), or a uniform disc
w(i, j) = 1 where (i^2 + j^2) p^2 <= R^2; output pixels whose support leaves the
map have no value (NaN); light curves interpolate bilinearly between pixel
centres at -L/2 + (I + 1/2) p.
"""
from __future__ import annotations

import math

import numpy as np


def profile_weights(profile: int, size_re: float, pix: float) -> np.ndarray:
    """Normalised (2h+1) x (2h+1) profile, index [dj + h, di + h]."""
    if profile == 0:
        h = math.ceil(4.0 * size_re / pix)
        k = np.arange(-h, h + 1) * pix
        g = np.exp(-k * k / (2.0 * size_re * size_re))
        w = np.outer(g, g)
    else:
        rp = size_re / pix
        h = int(math.floor(rp))
        k = np.arange(-h, h + 1)
        w = ((k[:, None] ** 2 + k[None, :] ** 2) <= rp * rp).astype(np.float64)
    return w / w.sum()


def convolve(counts, nrays: float, profile: int, size_re: float, pix: float) -> np.ndarray:
    """Direct sum over the profile's support, FP64; NaN where the support leaves the map."""
    mu = np.asarray(counts, dtype=np.float64) / nrays
    n = mu.shape[0]
    w = profile_weights(profile, size_re, pix)
    h = (w.shape[0] - 1) // 2
    out = np.full((n, n), np.nan)
    if 2 * h + 1 > n:
        return out
    acc = np.zeros((n - 2 * h, n - 2 * h))
    for dj in range(-h, h + 1):
        for di in range(-h, h + 1):
            wt = w[dj + h, di + h]
            if wt != 0.0:
                acc += wt * mu[h + dj:n - h + dj, h + di:n - h + di]
    out[h:n - h, h:n - h] = acc
    return out


def lightcurve(field, side: float, start, end, n_points: int) -> np.ndarray:
    """Bilinear samples of a convolved map along a straight source track."""
    n = field.shape[0]
    pix = side / n
    t = np.linspace(0.0, 1.0, n_points) if n_points > 1 else np.zeros(1)
    out = np.full(n_points, np.nan)
    for k, tk in enumerate(t):
        y1 = start[0] + tk * (end[0] - start[0])
        y2 = start[1] + tk * (end[1] - start[1])
        u = (y1 + side / 2) / pix - 0.5
        v = (y2 + side / 2) / pix - 0.5
        i, j = math.floor(u), math.floor(v)
        if u < 0 or v < 0 or i + 1 >= n or j + 1 >= n:
            continue
        a, b = u - i, v - j
        out[k] = ((1 - a) * (1 - b) * field[j, i] + a * (1 - b) * field[j, i + 1]
                  + (1 - a) * b * field[j + 1, i] + a * b * field[j + 1, i + 1])
    return out
