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


def convolve_at(counts, nrays: float, profile: int, size_re: float, pix: float, ii, jj) -> np.ndarray:
    """The convolved map of convolve() at pixels (ii[k], jj[k]) (column, row) only: the same direct
    FP64 sum of weight times mu over the profile's support, NaN where the support leaves the map. For
    maps too large to convolve whole in the oracle."""
    c = np.asarray(counts)
    n = c.shape[0]
    w = profile_weights(profile, size_re, pix)
    h = (w.shape[0] - 1) // 2
    out = np.full(len(ii), np.nan)
    for k, (i, j) in enumerate(zip(np.asarray(ii, dtype=np.int64), np.asarray(jj, dtype=np.int64))):
        if i - h < 0 or i + h >= n or j - h < 0 or j + h >= n:
            continue
        block = c[j - h:j + h + 1, i - h:i + h + 1].astype(np.float64) / nrays
        out[k] = float(np.sum(w * block))
    return out


def _track(n: int, side: float, start, end, n_points: int):
    """Samples of a straight track: pixel (i, j) below and left of each sample (pixel centres at
    -side/2 + (I + 1/2) side/n), bilinear weights (a, b), and whether all four pixels lie in the map."""
    pix = side / n
    t = np.linspace(0.0, 1.0, n_points) if n_points > 1 else np.zeros(1)
    out = []
    for tk in t:
        y1 = start[0] + tk * (end[0] - start[0])
        y2 = start[1] + tk * (end[1] - start[1])
        u = (y1 + side / 2) / pix - 0.5
        v = (y2 + side / 2) / pix - 0.5
        i, j = math.floor(u), math.floor(v)
        ok = not (u < 0 or v < 0 or i + 1 >= n or j + 1 >= n)
        out.append((i, j, u - i, v - j, ok))
    return out


def _bilinear(a, b, f00, f10, f01, f11):
    return (1 - a) * (1 - b) * f00 + a * (1 - b) * f10 + (1 - a) * b * f01 + a * b * f11


def lightcurve(field, side: float, start, end, n_points: int) -> np.ndarray:
    """Bilinear samples of a convolved map along a straight source track."""
    n = field.shape[0]
    out = np.full(n_points, np.nan)
    for k, (i, j, a, b, ok) in enumerate(_track(n, side, start, end, n_points)):
        if ok:
            out[k] = _bilinear(a, b, field[j, i], field[j, i + 1], field[j + 1, i], field[j + 1, i + 1])
    return out


def lightcurve_of_counts(counts, nrays: float, profile: int, size_re: float, side: float, start, end,
                         n_points: int) -> np.ndarray:
    """lightcurve() of the convolved map of counts, with only the four pixels each sample needs
    convolved (convolve_at): the same samples for maps too large to convolve whole."""
    n = np.asarray(counts).shape[0]
    samples = _track(n, side, start, end, n_points)
    ii, jj = [], []
    for i, j, _, _, ok in samples:
        if ok:
            ii += [i, i + 1, i, i + 1]
            jj += [j, j, j + 1, j + 1]
    f = convolve_at(counts, nrays, profile, size_re, side / n, ii, jj)
    out = np.full(n_points, np.nan)
    q = 0
    for k, (i, j, a, b, ok) in enumerate(samples):
        if ok:
            out[k] = _bilinear(a, b, *f[q:q + 4])
            q += 4
    return out
