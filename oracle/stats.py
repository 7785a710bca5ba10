"""Map statistics of the oracle (TEST INFRASTRUCTURE; see the package docstring).

Sect. 3.1: maps are compared by the root-mean-square difference of
Delta m = -2.5 log10(mu) (Eq. deltam, mu = N / N_rays per pixel) and by a
two-sample Kolmogorov-Smirnov test on the Delta m distributions. Readings:
the RMS runs over pixels where both maps count at least one ray; empty pixels
enter the K-S test with Delta m = +infinity; the K-S probability is the
asymptotic Kolmogorov distribution at (sqrt(n_e) + 0.12 + 0.11/sqrt(n_e)) D,
n_e = n_a n_b / (n_a + n_b). Written from these definitions with numpy and
scipy primitives (the empirical CDFs by sorting, the Kolmogorov survival
function from scipy.special).
"""
from __future__ import annotations

import numpy as np
from scipy.special import kolmogorov


def delta_m(counts, nrays):
    """Eq. deltam: -2.5 log10(N / N_rays); +inf for empty pixels."""
    c = np.asarray(counts, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return -2.5 * np.log10(c / nrays)


def ks_statistic(x, y):
    """Two-sample K-S statistic: max |F_x(t) - F_y(t)| over all sample values t."""
    x = np.sort(np.asarray(x, dtype=np.float64).ravel())
    y = np.sort(np.asarray(y, dtype=np.float64).ravel())
    t = np.concatenate([x, y])
    fx = np.searchsorted(x, t, side="right") / x.size
    fy = np.searchsorted(y, t, side="right") / y.size
    return float(np.max(np.abs(fx - fy)))


def ks_probability(d, na, nb):
    ne = na * nb / (na + nb)
    s = np.sqrt(ne)
    return float(kolmogorov((s + 0.12 + 0.11 / s) * d))


def compare(counts_a, nrays_a, counts_b, nrays_b) -> dict:
    a = np.asarray(counts_a).ravel()
    b = np.asarray(counts_b).ravel()
    da, db = delta_m(a, nrays_a), delta_m(b, nrays_b)
    both = (a > 0) & (b > 0)
    diff = da[both] - db[both]
    rms = float(np.sqrt(np.mean(diff * diff))) if both.any() else 0.0
    d = ks_statistic(da, db)
    return dict(rms_dm=rms, n_rms=int(both.sum()), zero_a=int((a == 0).sum()), zero_b=int((b == 0).sum()),
                ks_d=d, ks_p=ks_probability(d, a.size, b.size),
                mean_mu_a=float(a.sum() / (a.size * nrays_a)), mean_mu_b=float(b.sum() / (b.size * nrays_b)))
