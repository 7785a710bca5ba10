"""Each plausible mistake planted in a copy of the oracle must fail at least one pin.

The copy is built in a temporary directory on the CPU; the real oracle is
never modified. This shows that the pins in test_oracle_pins.py constrain
every term of the lens equation, the lattice, the binning and the layout,
those in test_oracle_far.py the far-field series, those in
test_oracle_stats.py the K-S probability of the map statistics, and those in
test_oracle_random_rays.py the random ray positions.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("smooth term sign", "- sigma_c * x1 - a1", "+ sigma_c * x1 - a1"),
    ("shear dropped on axis 1", "(1.0 - P->gamma) * x1", "(1.0) * x1"),
    ("shear sign on axis 2", "(1.0 + P->gamma) * x2", "(1.0 - P->gamma) * x2"),
    ("mass ignored", "s1 += lm[i] * d1 / r2;", "s1 += d1 / r2;"),
    ("lattice offset", "(double)i + 0.5 - 0.5", "(double)i - 0.5"),
    ("round instead of floor", "floor((y1 + 0.5 * P->side) / G->pix)", "floor((y1 + 0.5 * P->side) / G->pix + 0.5)"),
    ("transposed map", "return (int64_t)u2 * P->npix_side + (int64_t)u1;", "return (int64_t)u1 * P->npix_side + (int64_t)u2;"),
    ("deflection sign", "double y1 = (1.0 - P->gamma) * x1 - sigma_c * x1 - a1;",
     "double y1 = (1.0 - P->gamma) * x1 - sigma_c * x1 + a1;"),
    ("r^2 typo", "double r2 = d1 * d1 + d2 * d2;", "double r2 = d1 * d1 + d1 * d2;"),
    ("ray spacing", "G->delta = G->pix / sqrt(P->nrays);", "G->delta = G->pix / P->nrays;"),
    ("grid size", "G->nx = (int64_t)ceil(G->width / G->delta);", "G->nx = (int64_t)floor(G->width / G->delta);"),
    ("wrong component", "s2 += lm[i] * d2 / r2;", "s2 += lm[i] * d1 / r2;"),
]
PINS = "tests/test_oracle_pins.py"

# far-field approximation (Sect. 2.1, Eq. hierarchical), pinned by test_oracle_far.py
FAR = "tests/test_oracle_far.py"
FAR_MUTATIONS = [
    ("far series sign", "double complex t = -lm[i] * u;", "double complex t = lm[i] * u;"),
    ("far series power", "        t *= u;\n", "        t *= u * u;\n"),
    ("far series index shift", "f += B->c[l] * wl;", "f += B->c[l] * wl * w;"),
    ("far conjugate dropped", "*a2 = -cimag(f) + s2;", "*a2 = cimag(f) + s2;"),
    ("near radius squared twice", "return d1 * d1 + d2 * d2 < rn * rn;", "return d1 * d1 + d2 * d2 < rn;"),
    ("near lenses dropped", "for (int64_t k = 0; k < B->nnear; ++k)", "for (int64_t k = 0; k < 0; ++k)"),
    ("tail bound exponent", "pow(t, F->order)", "pow(t, F->order + 1)"),
    ("block radius halved", "B->rho = G->delta * sqrt(", "B->rho = 0.5 * G->delta * sqrt("),
    # grouped far lenses: the lens tree, the cells' expansions and their bound
    ("group binomial index", "binom[(l + q) * 130 + q]", "binom[(l + q + 1) * 130 + q]"),
    ("group sign alternation dropped", "const double sg = (q & 1) ? 1.0 : -1.0;", "const double sg = -1.0;"),
    ("group moments about the origin", "(lx[i] - N->xc) + I * (ly[i] - N->yc)", "lx[i] + I * ly[i]"),
    ("group power off by one", "up[l + q + 1]", "up[l + q]"),
    ("grouping ignores the near radius", "if (dabs - N->rc >= rn && ", "if ("),
    ("group bound drops the l >= P tail", "double e = pow(x / (1.0 - y), F->order) / (1.0 - x - y);",
     "double e = 0.0;"),
    ("tree loses a lens in a split", "part[k][cnt[k]++] = i;", "if (q > 0) part[k][cnt[k]++] = i;"),
    ("cell radius halved", "N->rc = s * 0.70710678118654752440;", "N->rc = s * 0.35355339059327376220;"),
]


# map statistics (Sect. 3.1): the K-S probability, pinned by test_oracle_stats.py
STATS = "tests/test_oracle_stats.py"
STATS_MUTATIONS = [
    ("K-S n_e as the sum of the sizes", "ne = na * nb / (na + nb)", "ne = na + nb"),
    ("K-S n_e as the smaller size", "ne = na * nb / (na + nb)", "ne = min(na, nb)"),
    ("K-S correction dropped", "kolmogorov((s + 0.12 + 0.11 / s) * d)", "kolmogorov(s * d)"),
    ("K-S 0.11/sqrt(n_e) term dropped", "kolmogorov((s + 0.12 + 0.11 / s) * d)", "kolmogorov((s + 0.12) * d)"),
    ("K-S 0.11 * sqrt(n_e) instead of 0.11/sqrt(n_e)", "kolmogorov((s + 0.12 + 0.11 / s) * d)",
     "kolmogorov((s + 0.12 + 0.11 * s) * d)"),
]

# random rays (Sect. 2.3, step 2), pinned by test_oracle_random_rays.py
RANDOM = "tests/test_oracle_random_rays.py"
RANDOM_MUTATIONS = [
    ("random stream shifted", "splitmix64_output(P->ray_seed, 2 * q + 1)", "splitmix64_output(P->ray_seed, 2 * q)"),
    ("random draws shared by the two axes", "splitmix64_output(P->ray_seed, 2 * q + 2)",
     "splitmix64_output(P->ray_seed, 2 * q + 1)"),
    ("random fraction from the wrong bits", "2 * q + 1) >> 46)", "2 * q + 1) >> 40)"),
    ("random tiles 64 rows high", "tj = j / 32;", "tj = j / 64;"),
    ("partial tile taken as whole", "G->nx - 64 * ti < 64 ? G->nx - 64 * ti : 64", "64"),
    ("random finaliser step dropped", "z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;", ""),
    ("random counter per ray index only", "(uint64_t)j * (uint64_t)G->nx + (uint64_t)i", "(uint64_t)i"),
]

CASES = ([m + (PINS, "mm_oracle.c") for m in MUTATIONS] + [m + (FAR, "mm_oracle.c") for m in FAR_MUTATIONS]
         + [m + (STATS, "stats.py") for m in STATS_MUTATIONS] + [m + (RANDOM, "mm_oracle.c") for m in RANDOM_MUTATIONS])


@pytest.mark.parametrize("name,old,new,pins,target", CASES, ids=[c[0] for c in CASES])
def test_pins_catch_planted_mistake(tmp_path, name, old, new, pins, target):
    for d in ("oracle", "synth", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("_build", "__pycache__", "*.so"))
    src = tmp_path / "oracle" / target
    text = src.read_text()
    assert text.count(old) == 1, f"mutation site not found: {old}"
    src.write_text(text.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        pins], cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"planted mistake '{name}' was not caught:\n{r.stdout[-2000:]}"
    assert "FAILED" in r.stdout
