/*
 * mm_oracle.c -- plain FP64 CPU oracle for direct inverse ray-shooting of
 * microlensing magnification maps.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this code; the library never does.
 *
 * It is the definition of the map written out, with no blocking, fusion or
 * reordering beyond what the definition states:
 *
 *   Lens equation with point masses, smooth matter and external shear
 *   (Sect. 2, Eq. sigma):
 *       y1 = (1 - gamma) x1 - sigma_c x1 - sum_i m_i (x1 - x1_i) / |x - x_i|^2
 *       y2 = (1 + gamma) x2 - sigma_c x2 - sum_i m_i (x2 - x2_i) / |x - x_i|^2
 *   with sigma_c = s * sigma (smooth fraction s = sigma_c / sigma, Sect. 3.1).
 *
 *   Inverse ray-shooting estimator (Sect. 2, the paragraph before Eq. sigma):
 *   rays are shot backwards from a regular image-plane grid (Sect. 3.1,
 *   regular grid of CPU-T) and counted into the source-plane pixel they land
 *   in; mu_ij = N_ij / N_rays, N_rays being the mean number of rays per
 *   pixel without lensing.
 *
 *   Shooting-grid geometry (Sect. 3.2.2, Eq. square): the source square of
 *   side L maps back to a rectangle of sides L/|1-sigma-gamma| and
 *   L/|1-sigma+gamma|. Readings taken where the paper is silent:
 *     - the shot rectangle is `margin` times that rectangle per side,
 *       centred on the origin;
 *     - rays lie on a square lattice of spacing Delta = p / sqrt(N_rays),
 *       p = L / N_side the pixel size, so that the unlensed ray density is
 *       N_rays per pixel; nx = ceil(W / Delta), ny = ceil(H / Delta);
 *       ray (i, j) sits at x1 = (i + 1/2 - nx/2) Delta,
 *       x2 = (j + 1/2 - ny/2) Delta (cell-centred, symmetric);
 *     - pixel (I, J) = (floor((y1 + L/2) / p), floor((y2 + L/2) / p)); a ray
 *       is counted iff 0 <= I, J < N_side, into counts[J * N_side + I]
 *       (row-major, row J along y2); otherwise it is "out";
 *     - a ray exactly on a lens (|x - x_i|^2 == 0) and any non-finite
 *       source position is "out".
 *   Lenses are summed in index order.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "mm_oracle.h"

/* Mean-field Jacobian diagonal: a = 1 - sigma - gamma, b = 1 - sigma + gamma
 * (Eq. sigma averaged over a uniform star field; Eq. square). */
int orc_geometry(const orc_params *P, orc_geometry_t *G)
{
    if (!P || !G) return -1;
    if (!(P->side > 0) || P->npix_side <= 0 || !(P->nrays > 0) || !(P->margin > 0)) return -1;
    double a = 1.0 - P->sigma - P->gamma;
    double b = 1.0 - P->sigma + P->gamma;
    if (fabs(a) < 1e-3 || fabs(b) < 1e-3) return -1;      /* Eq. square diverges */
    G->pix = P->side / (double)P->npix_side;
    G->delta = G->pix / sqrt(P->nrays);
    G->width = P->margin * P->side / fabs(a);
    G->height = P->margin * P->side / fabs(b);
    G->nx = (int64_t)ceil(G->width / G->delta);
    G->ny = (int64_t)ceil(G->height / G->delta);
    return 0;
}

/* Image-plane position of ray (i, j) on the regular grid. */
static void ray_position(const orc_geometry_t *G, int64_t i, int64_t j, double *x1, double *x2)
{
    *x1 = ((double)i + 0.5 - 0.5 * (double)G->nx) * G->delta;
    *x2 = ((double)j + 0.5 - 0.5 * (double)G->ny) * G->delta;
}

/* Star deflection alpha(x) = sum_i m_i (x - x_i) / |x - x_i|^2 (Eq. sigma).
 * Returns 0, or 1 if the ray sits exactly on a lens. */
static int deflection(const double *lx, const double *ly, const double *lm, int64_t nstar,
                      double x1, double x2, double *a1, double *a2)
{
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = 0; i < nstar; ++i) {
        double d1 = x1 - lx[i];
        double d2 = x2 - ly[i];
        double r2 = d1 * d1 + d2 * d2;
        if (r2 == 0.0) return 1;
        s1 += lm[i] * d1 / r2;
        s2 += lm[i] * d2 / r2;
    }
    *a1 = s1;
    *a2 = s2;
    return 0;
}

/* Source position and pixel of one ray; returns the flat pixel index or -1 (out). */
static int64_t shoot_one(const orc_params *P, const orc_geometry_t *G,
                         const double *lx, const double *ly, const double *lm, int64_t nstar,
                         int64_t i, int64_t j, double *alpha, double *ysrc)
{
    double x1, x2, a1 = NAN, a2 = NAN;
    ray_position(G, i, j, &x1, &x2);
    int on_lens = deflection(lx, ly, lm, nstar, x1, x2, &a1, &a2);
    double sigma_c = P->smooth_frac * P->sigma;
    double y1 = (1.0 - P->gamma) * x1 - sigma_c * x1 - a1;
    double y2 = (1.0 + P->gamma) * x2 - sigma_c * x2 - a2;
    if (alpha) { alpha[0] = a1; alpha[1] = a2; }
    if (ysrc) { ysrc[0] = y1; ysrc[1] = y2; }
    if (on_lens || !isfinite(y1) || !isfinite(y2)) return -1;
    double u1 = floor((y1 + 0.5 * P->side) / G->pix);
    double u2 = floor((y2 + 0.5 * P->side) / G->pix);
    if (u1 < 0.0 || u2 < 0.0 || u1 >= (double)P->npix_side || u2 >= (double)P->npix_side) return -1;
    return (int64_t)u2 * P->npix_side + (int64_t)u1;
}

int orc_map(const orc_params *P, const double *lx, const double *ly, const double *lm, int64_t nstar,
            int64_t i0, int64_t i1, int64_t j0, int64_t j1, int64_t stride,
            uint32_t *counts, uint64_t totals[3], int nthreads)
{
    orc_geometry_t G;
    if (orc_geometry(P, &G) != 0 || !counts || !totals || nstar < 0 || stride <= 0) return -1;
    if (nstar > 0 && (!lx || !ly || !lm)) return -1;
    if (i0 < 0) { i0 = 0; i1 = G.nx; j0 = 0; j1 = G.ny; }
    if (i1 > G.nx) i1 = G.nx;
    if (j1 > G.ny) j1 = G.ny;
    size_t npix = (size_t)P->npix_side * (size_t)P->npix_side;
    memset(counts, 0, npix * sizeof(uint32_t));
    uint64_t shot = 0, in = 0, out = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel for schedule(dynamic, 1) reduction(+:shot, in, out)
    for (int64_t j = j0; j < j1; j += stride) {
        for (int64_t i = i0; i < i1; i += stride) {
            int64_t k = shoot_one(P, &G, lx, ly, lm, nstar, i, j, NULL, NULL);
            shot += 1;
            if (k >= 0) {
                #pragma omp atomic update
                counts[k] += 1u;
                in += 1;
            } else {
                out += 1;
            }
        }
    }
    totals[0] = shot;
    totals[1] = in;
    totals[2] = out;
    return 0;
}

int orc_rays(const orc_params *P, const double *lx, const double *ly, const double *lm, int64_t nstar,
             const int64_t *ray_i, const int64_t *ray_j, int64_t n,
             double *alpha, double *ysrc, int64_t *pixel, int nthreads)
{
    orc_geometry_t G;
    if (orc_geometry(P, &G) != 0 || n < 0 || !ray_i || !ray_j || !alpha || !ysrc || !pixel) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k)
        pixel[k] = shoot_one(P, &G, lx, ly, lm, nstar, ray_i[k], ray_j[k], alpha + 2 * k, ysrc + 2 * k);
    return 0;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
