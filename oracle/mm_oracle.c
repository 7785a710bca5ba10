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
 *
 * The far-field approximation (orc_far_map, orc_far_rays) is at the end of
 * this file, with its own statement.
 */
#include <complex.h>
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

/* Add lens i's term m_i (x - x_i) / |x - x_i|^2 of Eq. sigma to (s1, s2).
 * Returns 1 (and adds nothing) if the ray sits exactly on the lens. */
static int add_lens(const double *lx, const double *ly, const double *lm, int64_t i, double x1, double x2,
                    double *s1, double *s2)
{
    double d1 = x1 - lx[i];
    double d2 = x2 - ly[i];
    double r2 = d1 * d1 + d2 * d2;
    if (r2 == 0.0) return 1;
    *s1 += lm[i] * d1 / r2;
    *s2 += lm[i] * d2 / r2;
    return 0;
}

/* Star deflection alpha(x) = sum_i m_i (x - x_i) / |x - x_i|^2 (Eq. sigma).
 * Returns 0, or 1 if the ray sits exactly on a lens. */
static int deflection(const double *lx, const double *ly, const double *lm, int64_t nstar,
                      double x1, double x2, double *a1, double *a2)
{
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = 0; i < nstar; ++i)
        if (add_lens(lx, ly, lm, i, x1, x2, &s1, &s2)) return 1;
    *a1 = s1;
    *a2 = s2;
    return 0;
}

/* Lens equation (Eq. sigma) and binning of a ray at (x1, x2) with star deflection
 * (a1, a2); returns the flat pixel index or -1 (out). */
static int64_t source_pixel(const orc_params *P, const orc_geometry_t *G, double x1, double x2, double a1, double a2,
                            int on_lens, double *alpha, double *ysrc)
{
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

/* Source position and pixel of one ray; returns the flat pixel index or -1 (out). */
static int64_t shoot_one(const orc_params *P, const orc_geometry_t *G,
                         const double *lx, const double *ly, const double *lm, int64_t nstar,
                         int64_t i, int64_t j, double *alpha, double *ysrc)
{
    double x1, x2, a1 = NAN, a2 = NAN;
    ray_position(G, i, j, &x1, &x2);
    int on_lens = deflection(lx, ly, lm, nstar, x1, x2, &a1, &a2);
    return source_pixel(P, G, x1, x2, a1, a2, on_lens, alpha, ysrc);
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

/* ===========================================================================
 * Far-field approximation (the tree code's idea, Sect. 2.1, Eq. hierarchical).
 *
 * The paper's tree code sums near lenses one by one and replaces groups of
 * distant lenses by pseudo-lenses. The pseudo-lens deflection is computed only
 * for "test rays" and interpolated for the rays around them. Here the rays are
 * grouped into blocks, and the block centre plays the test ray:
 *
 *   - Blocks. The shot rectangle, from its origin (i0, j0), is cut into blocks
 *     of 64 bt x 32 bt rays. Block (BX, BY) holds rays
 *     i in [i0 + 64 bt BX, i0 + 64 bt (BX + 1)), j likewise with 32 bt. Its
 *     centre z_B is the centre of those lattice cells. Its radius
 *     rho = Delta sqrt((32 bt)^2 + (16 bt)^2) exceeds |z - z_B| for every
 *     ray z of the block.
 *   - Near and far. With d_i = z_i - z_B, lens i is near iff
 *     |d_i|^2 < (rho / q)^2. Near lenses are summed exactly, as in Eq. sigma.
 *   - Far series. In complex notation, the star deflection obeys
 *     conj(alpha(z)) = sum_i m_i / (z - z_i). For a far lens,
 *     1 / (z - z_i) = -sum_l w^l / d_i^(l+1) with w = z - z_B, because
 *     |w| < |d_i|. Keeping P terms, the far lenses' contribution is
 *     sum_{l<P} c_l w^l, with c_l = -sum_{far i} m_i d_i^-(l+1).
 *   - Bound. The truncation error is at most
 *     sum_{far i} m_i t_i^P / (|d_i| (1 - t_i)), with t_i = |w| / |d_i| < q.
 *     This is the tail of the geometric series.
 *
 * P = 1 keeps only c_0: the far lenses' deflection at the test ray, unchanged
 * across the block. A ratio q so small that every lens is near gives the
 * direct sum of Eq. sigma back, bit for bit.
 * ======================================================================== */

typedef struct {
    double xb, yb;          /* block centre z_B */
    double rho;             /* block radius */
    int64_t nnear;
    int64_t *near;          /* near lens indices, ascending */
    char *is_near;          /* [nstar] */
    double complex *c;      /* [P] far-series coefficients */
} far_block;

static int far_params_ok(const orc_far_params *F)
{
    return F && F->order >= 1 && F->order <= 64 && F->ratio > 0.0 && F->ratio < 1.0 && F->block_tiles >= 1;
}

static void far_block_free(far_block *B)
{
    free(B->near);
    free(B->is_near);
    free(B->c);
}

/* Block (BX, BY) of the rectangle with origin (i0, j0): centre, near list and series. */
static int far_block_build(const orc_far_params *F, const orc_geometry_t *G, const double *lx, const double *ly,
                           const double *lm, int64_t nstar, int64_t i0, int64_t j0, int64_t BX, int64_t BY,
                           far_block *B)
{
    const int64_t bw = 64 * (int64_t)F->block_tiles, bh = 32 * (int64_t)F->block_tiles;
    B->xb = ((double)(i0 + BX * bw + bw / 2) - 0.5 * (double)G->nx) * G->delta;
    B->yb = ((double)(j0 + BY * bh + bh / 2) - 0.5 * (double)G->ny) * G->delta;
    B->rho = G->delta * sqrt((double)(bw / 2) * (double)(bw / 2) + (double)(bh / 2) * (double)(bh / 2));
    const double rn = B->rho / F->ratio;
    B->nnear = 0;
    B->near = (int64_t *)malloc((size_t)(nstar > 0 ? nstar : 1) * sizeof(int64_t));
    B->is_near = (char *)calloc((size_t)(nstar > 0 ? nstar : 1), 1);
    B->c = (double complex *)calloc((size_t)F->order, sizeof(double complex));
    if (!B->near || !B->is_near || !B->c) {
        far_block_free(B);
        return -1;
    }
    for (int64_t i = 0; i < nstar; ++i) {
        const double d1 = lx[i] - B->xb, d2 = ly[i] - B->yb;
        if (d1 * d1 + d2 * d2 < rn * rn) {
            B->near[B->nnear++] = i;
            B->is_near[i] = 1;
            continue;
        }
        const double complex u = 1.0 / (d1 + I * d2);           /* 1 / d_i */
        double complex t = -lm[i] * u;                          /* -m_i / d_i^(l+1) for l = 0 */
        for (int l = 0; l < F->order; ++l) {
            B->c[l] += t;
            t *= u;
        }
    }
    return 0;
}

/* Truncation bound at offset |w| from the block centre. */
static double far_bound(const far_block *B, const orc_far_params *F, const double *lx, const double *ly,
                        const double *lm, int64_t nstar, double wabs)
{
    double b = 0.0;
    for (int64_t i = 0; i < nstar; ++i) {
        if (B->is_near[i]) continue;
        const double d = hypot(lx[i] - B->xb, ly[i] - B->yb);
        const double t = wabs / d;
        b += lm[i] * pow(t, F->order) / (d * (1.0 - t));
    }
    return b;
}

/* Deflection of ray (i, j) of block B: the far series at w plus the near lenses in
 * index order. Returns 1 if the ray sits exactly on a near lens. */
static int far_deflection(const far_block *B, const orc_far_params *F, const double *lx, const double *ly,
                          const double *lm, double x1, double x2, double *a1, double *a2)
{
    const double complex w = (x1 - B->xb) + I * (x2 - B->yb);
    double complex f = 0.0, wl = 1.0;
    for (int l = 0; l < F->order; ++l) {
        f += B->c[l] * wl;
        wl *= w;
    }
    double s1 = 0.0, s2 = 0.0;
    for (int64_t k = 0; k < B->nnear; ++k)
        if (add_lens(lx, ly, lm, B->near[k], x1, x2, &s1, &s2)) return 1;
    *a1 = creal(f) + s1;          /* alpha = conj(f) + near sum */
    *a2 = -cimag(f) + s2;
    return 0;
}

int orc_far_map(const orc_params *P, const orc_far_params *F, const double *lx, const double *ly, const double *lm,
                int64_t nstar, int64_t i0, int64_t i1, int64_t j0, int64_t j1,
                uint32_t *counts, uint64_t totals[3], double *bound_max, int nthreads)
{
    orc_geometry_t G;
    if (orc_geometry(P, &G) != 0 || !far_params_ok(F) || !counts || !totals || nstar < 0) return -1;
    if (nstar > 0 && (!lx || !ly || !lm)) return -1;
    if (i0 < 0) { i0 = 0; i1 = G.nx; j0 = 0; j1 = G.ny; }
    if (i1 > G.nx) i1 = G.nx;
    if (j1 > G.ny) j1 = G.ny;
    if (i1 < i0 || j1 < j0) return -1;
    const int64_t bw = 64 * (int64_t)F->block_tiles, bh = 32 * (int64_t)F->block_tiles;
    const int64_t nbx = (i1 - i0 + bw - 1) / bw, nby = (j1 - j0 + bh - 1) / bh;
    memset(counts, 0, (size_t)P->npix_side * (size_t)P->npix_side * sizeof(uint32_t));
    uint64_t shot = 0, in = 0, out = 0;
    double bmax = 0.0;
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel for schedule(dynamic, 1) reduction(+:shot, in, out, err) reduction(max:bmax)
    for (int64_t b = 0; b < nbx * nby; ++b) {
        const int64_t BX = b % nbx, BY = b / nbx;
        far_block B;
        if (far_block_build(F, &G, lx, ly, lm, nstar, i0, j0, BX, BY, &B) != 0) {
            err += 1;
            continue;
        }
        const double bb = far_bound(&B, F, lx, ly, lm, nstar, B.rho);
        if (bb > bmax) bmax = bb;
        const int64_t ie = i0 + (BX + 1) * bw < i1 ? i0 + (BX + 1) * bw : i1;
        const int64_t je = j0 + (BY + 1) * bh < j1 ? j0 + (BY + 1) * bh : j1;
        for (int64_t j = j0 + BY * bh; j < je; ++j) {
            for (int64_t i = i0 + BX * bw; i < ie; ++i) {
                double x1, x2, a1 = NAN, a2 = NAN;
                ray_position(&G, i, j, &x1, &x2);
                const int on_lens = far_deflection(&B, F, lx, ly, lm, x1, x2, &a1, &a2);
                const int64_t k = source_pixel(P, &G, x1, x2, a1, a2, on_lens, NULL, NULL);
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
        far_block_free(&B);
    }
    if (err) return -1;
    totals[0] = shot;
    totals[1] = in;
    totals[2] = out;
    if (bound_max) *bound_max = bmax;
    return 0;
}

int orc_far_rays(const orc_params *P, const orc_far_params *F, const double *lx, const double *ly, const double *lm,
                 int64_t nstar, int64_t i0, int64_t j0, const int64_t *ray_i, const int64_t *ray_j, int64_t n,
                 double *alpha, double *ysrc, int64_t *pixel, double *bound, int nthreads)
{
    orc_geometry_t G;
    if (orc_geometry(P, &G) != 0 || !far_params_ok(F) || n < 0 || !ray_i || !ray_j || !alpha || !ysrc || !pixel ||
        !bound || i0 < 0 || j0 < 0)
        return -1;
    const int64_t bw = 64 * (int64_t)F->block_tiles, bh = 32 * (int64_t)F->block_tiles;
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    #pragma omp parallel for schedule(dynamic, 16) reduction(+:err)
    for (int64_t k = 0; k < n; ++k) {
        if (ray_i[k] < i0 || ray_j[k] < j0) {
            err += 1;
            continue;
        }
        far_block B;
        if (far_block_build(F, &G, lx, ly, lm, nstar, i0, j0, (ray_i[k] - i0) / bw, (ray_j[k] - j0) / bh, &B) != 0) {
            err += 1;
            continue;
        }
        double x1, x2, a1 = NAN, a2 = NAN;
        ray_position(&G, ray_i[k], ray_j[k], &x1, &x2);
        const int on_lens = far_deflection(&B, F, lx, ly, lm, x1, x2, &a1, &a2);
        pixel[k] = source_pixel(P, &G, x1, x2, a1, a2, on_lens, alpha + 2 * k, ysrc + 2 * k);
        bound[k] = far_bound(&B, F, lx, ly, lm, nstar, hypot(x1 - B.xb, x2 - B.yb));
        far_block_free(&B);
    }
    return err ? -1 : 0;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
