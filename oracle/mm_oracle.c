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
 *   Random rays (ray_mode ORC_RAYS_RANDOM): the paper's GPU code shoots rays from
 *   pseudo-random positions, so that a pixel receives N_rays rays on average only
 *   (Sect. 2.3, step 2; Sect. 3.1). Reading taken: the same nx * ny rays are shot,
 *   ray (i, j) uniformly at random in the 64 x 32-cell tile of the lattice that
 *   holds cell (i, j), independently of every other ray (see ray_position).
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

/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014): output k >= 1 of the generator seeded with s is mix(s + k * gamma mod 2^64),
 * gamma = 0x9E3779B97F4A7C15, with the finaliser mix(z): z ^= z >> 30, z *= 0xBF58476D1CE4E5B9,
 * z ^= z >> 27, z *= 0x94D049BB133111EB, z ^= z >> 31. */
static uint64_t splitmix64_output(uint64_t s, uint64_t k)
{
    uint64_t z = s + k * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Image-plane position of ray (i, j).
 * Lattice: the centre of cell (i, j).
 * Random: with q = j nx + i, u1 and u2 are the top 18 bits of outputs 2q + 1 and 2q + 2 of
 * SplitMix64(ray_seed), as fractions in [0, 1) (18 bits, so that u w below is exact in single
 * precision too); the tile is (Ti, Tj) = (floor(i / 64), floor(j / 32)), its width in cells
 * wi = min(64, nx - 64 Ti) and height wj = min(32, ny - 32 Tj), and the ray sits at
 *     x1 = (64 Ti + u1 wi - nx/2) Delta,   x2 = (32 Tj + u2 wj - ny/2) Delta,
 * so that every ray is uniform over its (possibly partial) tile and the shot rectangle keeps
 * the lattice's ray density. */
static void ray_position(const orc_params *P, const orc_geometry_t *G, int64_t i, int64_t j, double *x1,
                         double *x2)
{
    if (P->ray_mode != ORC_RAYS_RANDOM) {
        *x1 = ((double)i + 0.5 - 0.5 * (double)G->nx) * G->delta;
        *x2 = ((double)j + 0.5 - 0.5 * (double)G->ny) * G->delta;
        return;
    }
    const uint64_t q = (uint64_t)j * (uint64_t)G->nx + (uint64_t)i;
    const double u1 = (double)(splitmix64_output(P->ray_seed, 2 * q + 1) >> 46) / 262144.0;
    const double u2 = (double)(splitmix64_output(P->ray_seed, 2 * q + 2) >> 46) / 262144.0;
    const int64_t ti = i / 64, tj = j / 32;
    const int64_t wi = G->nx - 64 * ti < 64 ? G->nx - 64 * ti : 64;
    const int64_t wj = G->ny - 32 * tj < 32 ? G->ny - 32 * tj : 32;
    *x1 = ((double)(64 * ti) + u1 * (double)wi - 0.5 * (double)G->nx) * G->delta;
    *x2 = ((double)(32 * tj) + u2 * (double)wj - 0.5 * (double)G->ny) * G->delta;
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
    ray_position(P, G, i, j, &x1, &x2);
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
 *
 * Grouped far lenses (group_order K > 0): the tree code also groups distant
 * lenses into cells of a tree and lets each cell act through its multipole
 * moments. The statement used here:
 *
 *   - Lens tree. R0 is the smallest power of two above every |x_i| and |y_i|.
 *     Level L cuts the square [-R0, R0)^2 into 2^L x 2^L cells of side
 *     s_L = 2 R0 / 2^L; lens i lies in cell (floor((x_i + R0) / s_L),
 *     floor((y_i + R0) / s_L)) (each index capped at 2^L - 1). The root is the
 *     level-0 cell; a cell with more than group_leaf lenses, below level 16, has
 *     its non-empty sub-cells of the next level as children; other cells are
 *     leaves. A cell C has centre z_C (the square's centre), half-diagonal
 *     r_C = s_L / sqrt(2), and moments a_k = sum_{i in C} m_i (z_i - z_C)^k,
 *     k < K.
 *   - Grouping. For block B, a cell C with D = z_C - z_B is grouped when
 *     |D| - r_C >= rho / q (every lens of C is far) and rho + r_C <= theta |D|.
 *     The tree is walked from the root: a grouped cell adds
 *     c_l += -sum_{k<K} (-1)^k C(l+k, k) a_k / D^(l+k+1)
 *     (the series of 1 / (D + e)^(l+1) in e = z_i - z_C, term by term, summed
 *     over the cell's lenses); a leaf that is not grouped adds its lenses one
 *     by one (near or far, as above); any other cell passes to its children.
 *     The near lenses are therefore the same as without grouping.
 *   - Bound. For a lens of a grouped cell, the double series of
 *     1 / (w - D - e) in w and e has terms bounded by C(l+k, k) x^l y^k / |D|,
 *     x = |w| / |D|, y = |e| / |D| <= r_C / |D|, x + y < 1. The terms kept are
 *     l < P, k < K, so the cell adds at most
 *     (M_C / |D|) E(x, y), M_C = sum of its masses,
 *     E = (x / (1 - y))^P / (1 - x - y) + sum_{l<P} x^l sum_{k>=K} C(l+k, k) y^k,
 *     to the bound of the lenses taken one by one; the inner sum takes its first four terms
 *     and bounds the rest by a geometric series (binom_tail).
 * ======================================================================== */

#define TREE_LMAX 16

typedef struct {
    int level;
    double xc, yc;          /* cell centre z_C */
    double rc;              /* half-diagonal r_C */
    int64_t n;              /* lenses in the cell */
    int64_t *idx;           /* their indices, ascending */
    int child[4], nchild;   /* non-empty sub-cells; a leaf has none */
    double mass;            /* M_C */
    double complex *a;      /* [K] moments */
} tree_node;

typedef struct {
    tree_node *nodes;
    int nn, cap;
    double r0;
    int K;
} lens_tree;

typedef struct {
    double xb, yb;          /* block centre z_B */
    double rho;             /* block radius */
    int64_t nnear;
    int64_t *near;          /* near lens indices, ascending */
    int64_t nfar;
    int64_t *far;           /* lenses in the series one by one, ascending */
    int nacc;
    double *acc;            /* grouped cells: (M_C, |D|, r_C) triples */
    double complex *c;      /* [P] far-series coefficients */
} far_block;

static int far_params_ok(const orc_far_params *F)
{
    if (!F || F->order < 1 || F->order > 64 || !(F->ratio > 0.0) || !(F->ratio < 1.0) || F->block_tiles < 1)
        return 0;
    if (F->group_order < 0 || F->group_order > 64) return 0;
    if (F->group_order > 0 && (!(F->group_theta > 0.0) || !(F->group_theta < 1.0) || F->group_leaf < 1)) return 0;
    return 1;
}

static void far_block_free(far_block *B)
{
    free(B->near);
    free(B->far);
    free(B->acc);
    free(B->c);
}

/* Smallest power of two above every |x_i| and |y_i| (1 for no lenses or all at the origin). */
static double tree_root_half(const double *lx, const double *ly, int64_t n)
{
    double m = 0.0;
    for (int64_t i = 0; i < n; ++i) m = fmax(m, fmax(fabs(lx[i]), fabs(ly[i])));
    if (m == 0.0) return 1.0;
    int e;
    frexp(m, &e);                    /* m = f 2^e, 1/2 <= f < 1 */
    return ldexp(1.0, e);
}

/* Cell index of coordinate v at level L (cells of side s from -R0). */
static int64_t cell_index(double v, double r0, double s, int level)
{
    int64_t c = (int64_t)floor((v + r0) / s);
    const int64_t top = ((int64_t)1 << level) - 1;
    return c < 0 ? 0 : (c > top ? top : c);
}

static void tree_free(lens_tree *T)
{
    for (int k = 0; k < T->nn; ++k) {
        free(T->nodes[k].idx);
        free(T->nodes[k].a);
    }
    free(T->nodes);
    T->nodes = NULL;
    T->nn = T->cap = 0;
}

/* Add the cell (level, ix, iy) holding lenses idx[0..n) (ascending, taken over by the
 * node) and its subtree; returns its node index, or -1 when memory runs out. */
static int tree_add(lens_tree *T, int level, int64_t ix, int64_t iy, int64_t *idx, int64_t n, const double *lx,
                    const double *ly, const double *lm, int leaf)
{
    if (T->nn == T->cap) {
        const int cap = T->cap ? 2 * T->cap : 64;
        tree_node *p = (tree_node *)realloc(T->nodes, (size_t)cap * sizeof(tree_node));
        if (!p) { free(idx); return -1; }
        T->nodes = p;
        T->cap = cap;
    }
    const int me = T->nn++;
    tree_node *N = &T->nodes[me];
    memset(N, 0, sizeof(*N));
    const double s = ldexp(T->r0, 1 - level);
    N->level = level;
    N->xc = -T->r0 + ((double)ix + 0.5) * s;
    N->yc = -T->r0 + ((double)iy + 0.5) * s;
    N->rc = s * 0.70710678118654752440;
    N->n = n;
    N->idx = idx;
    N->a = (double complex *)calloc((size_t)T->K, sizeof(double complex));
    if (!N->a) return -1;
    for (int64_t q = 0; q < n; ++q) {
        const int64_t i = idx[q];
        const double complex e = (lx[i] - N->xc) + I * (ly[i] - N->yc);
        double complex pw = 1.0;
        N->mass += lm[i];
        for (int k = 0; k < T->K; ++k) {
            N->a[k] += lm[i] * pw;
            pw *= e;
        }
    }
    if (n <= leaf || level >= TREE_LMAX) return me;
    /* children: the sub-cells of level + 1, in the order (0,0), (1,0), (0,1), (1,1) */
    const double sc = ldexp(T->r0, -level);
    int64_t *part[4];
    int64_t cnt[4] = {0, 0, 0, 0};
    for (int q = 0; q < 4; ++q) {
        part[q] = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        if (!part[q]) { for (int r = 0; r < q; ++r) free(part[r]); return -1; }
    }
    for (int64_t q = 0; q < n; ++q) {
        const int64_t i = idx[q];
        const int64_t cx = cell_index(lx[i], T->r0, sc, level + 1) - 2 * ix;
        const int64_t cy = cell_index(ly[i], T->r0, sc, level + 1) - 2 * iy;
        const int k = (int)(cy * 2 + cx);
        part[k][cnt[k]++] = i;
    }
    for (int q = 0; q < 4; ++q) {
        if (cnt[q] == 0) { free(part[q]); continue; }
        const int ch = tree_add(T, level + 1, 2 * ix + (q & 1), 2 * iy + (q >> 1), part[q], cnt[q], lx, ly, lm, leaf);
        if (ch < 0) { for (int r = q + 1; r < 4; ++r) free(part[r]); return -1; }
        N = &T->nodes[me];                  /* the node array may have moved */
        N->child[N->nchild++] = ch;
    }
    return me;
}

static int tree_build(lens_tree *T, const orc_far_params *F, const double *lx, const double *ly, const double *lm,
                      int64_t nstar)
{
    memset(T, 0, sizeof(*T));
    T->K = F->group_order;
    if (T->K == 0 || nstar == 0) return 0;
    T->r0 = tree_root_half(lx, ly, nstar);
    int64_t *all = (int64_t *)malloc((size_t)nstar * sizeof(int64_t));
    if (!all) return -1;
    for (int64_t i = 0; i < nstar; ++i) all[i] = i;
    return tree_add(T, 0, 0, 0, all, nstar, lx, ly, lm, F->group_leaf) < 0 ? -1 : 0;
}

/* Lens at offset (d1, d2) from a block centre is near iff |d|^2 < (rho / q)^2. */
static int is_near(double d1, double d2, double rn)
{
    return d1 * d1 + d2 * d2 < rn * rn;
}

static int cmp_i64(const void *p, const void *q)
{
    const int64_t a = *(const int64_t *)p, b = *(const int64_t *)q;
    return (a > b) - (a < b);
}

/* Walk the tree for block B: grouped cells go to B->acc (and their series into c),
 * lenses of the other leaves to the near or the one-by-one list. */
static void tree_visit(const lens_tree *T, int k, const orc_far_params *F, const double *lx, const double *ly,
                       double rn, far_block *B, double complex *cg, const double *binom)
{
    const tree_node *N = &T->nodes[k];
    const double complex D = (N->xc - B->xb) + I * (N->yc - B->yb);
    const double dabs = cabs(D);
    if (dabs - N->rc >= rn && B->rho + N->rc <= F->group_theta * dabs) {
        const int P = F->order, K = T->K;
        const double complex u = 1.0 / D;
        double complex up[130];              /* u^j, j <= P + K */
        up[0] = 1.0;
        for (int j = 1; j <= P + K; ++j) up[j] = up[j - 1] * u;
        for (int l = 0; l < P; ++l)
            for (int q = 0; q < K; ++q) {
                const double sg = (q & 1) ? 1.0 : -1.0;           /* -(-1)^q */
                cg[l] += sg * binom[(l + q) * 130 + q] * N->a[q] * up[l + q + 1];
            }
        B->acc[3 * B->nacc] = N->mass;
        B->acc[3 * B->nacc + 1] = dabs;
        B->acc[3 * B->nacc + 2] = N->rc;
        B->nacc++;
        return;
    }
    if (N->nchild == 0) {
        for (int64_t q = 0; q < N->n; ++q) {
            const int64_t i = N->idx[q];
            if (is_near(lx[i] - B->xb, ly[i] - B->yb, rn)) B->near[B->nnear++] = i;
            else B->far[B->nfar++] = i;
        }
        return;
    }
    for (int q = 0; q < N->nchild; ++q) tree_visit(T, N->child[q], F, lx, ly, rn, B, cg, binom);
}

/* Pascal's triangle C(n, k), n, k < 130, row-major [n * 130 + k]. */
static double *binom_table(void)
{
    double *b = (double *)calloc(130 * 130, sizeof(double));
    if (!b) return NULL;
    for (int n = 0; n < 130; ++n) {
        b[n * 130] = 1.0;
        for (int k = 1; k <= n; ++k) b[n * 130 + k] = b[(n - 1) * 130 + k - 1] + (k < n ? b[(n - 1) * 130 + k] : 0.0);
    }
    return b;
}

/* Block (BX, BY) of the rectangle with origin (i0, j0): centre, near list and series. */
static int far_block_build(const orc_far_params *F, const orc_geometry_t *G, const lens_tree *T, const double *binom,
                           const double *lx, const double *ly, const double *lm, int64_t nstar, int64_t i0,
                           int64_t j0, int64_t BX, int64_t BY, far_block *B)
{
    const int64_t bw = 64 * (int64_t)F->block_tiles, bh = 32 * (int64_t)F->block_tiles;
    memset(B, 0, sizeof(*B));
    B->xb = ((double)(i0 + BX * bw + bw / 2) - 0.5 * (double)G->nx) * G->delta;
    B->yb = ((double)(j0 + BY * bh + bh / 2) - 0.5 * (double)G->ny) * G->delta;
    B->rho = G->delta * sqrt((double)(bw / 2) * (double)(bw / 2) + (double)(bh / 2) * (double)(bh / 2));
    const double rn = B->rho / F->ratio;
    const size_t cap = (size_t)(nstar > 0 ? nstar : 1);
    B->near = (int64_t *)malloc(cap * sizeof(int64_t));
    B->far = (int64_t *)malloc(cap * sizeof(int64_t));
    B->acc = (double *)malloc((size_t)(T->nn > 0 ? T->nn : 1) * 3 * sizeof(double));
    B->c = (double complex *)calloc((size_t)F->order, sizeof(double complex));
    double complex *cg = (double complex *)calloc((size_t)F->order, sizeof(double complex));
    if (!B->near || !B->far || !B->acc || !B->c || !cg) {
        free(cg);
        far_block_free(B);
        return -1;
    }
    if (T->nn > 0) {
        tree_visit(T, 0, F, lx, ly, rn, B, cg, binom);
        qsort(B->near, (size_t)B->nnear, sizeof(int64_t), cmp_i64);
        qsort(B->far, (size_t)B->nfar, sizeof(int64_t), cmp_i64);
    } else {
        for (int64_t i = 0; i < nstar; ++i) {
            if (is_near(lx[i] - B->xb, ly[i] - B->yb, rn)) B->near[B->nnear++] = i;
            else B->far[B->nfar++] = i;
        }
    }
    /* lenses one by one, in index order, then the grouped cells */
    for (int64_t q = 0; q < B->nfar; ++q) {
        const int64_t i = B->far[q];
        const double complex u = 1.0 / ((lx[i] - B->xb) + I * (ly[i] - B->yb));   /* 1 / d_i */
        double complex t = -lm[i] * u;                          /* -m_i / d_i^(l+1) for l = 0 */
        for (int l = 0; l < F->order; ++l) {
            B->c[l] += t;
            t *= u;
        }
    }
    for (int l = 0; l < F->order; ++l) B->c[l] += cg[l];
    free(cg);
    return 0;
}

/* sum_{k>=K} C(l+k, k) y^k: the first four terms exactly, then the rest by a geometric series
 * of the ratio of the last term kept to the one before -- the ratios y (l+k+1)/(k+1) fall with
 * k, so every later term is at most that ratio times the one before it. When that ratio is not
 * below 1 yet, more terms are kept until it is. */
static double binom_tail(int l, int K, double y, const double *binom)
{
    double term = binom[(l + K) * 130 + K] * pow(y, K);
    double sum = 0.0;
    for (int k = K; k < K + 100000; ++k) {
        sum += term;
        const double r = y * (double)(l + k + 1) / (double)(k + 1);       /* term(k+1) / term(k) */
        term *= r;
        if (k >= K + 3 && r < 1.0) return sum + term / (1.0 - r);
    }
    return INFINITY;
}

/* Truncation bound at offset |w| from the block centre. */
static double far_bound(const far_block *B, const orc_far_params *F, const double *binom, const double *lx,
                        const double *ly, const double *lm, double wabs)
{
    double b = 0.0;
    for (int64_t q = 0; q < B->nfar; ++q) {
        const int64_t i = B->far[q];
        const double d = hypot(lx[i] - B->xb, ly[i] - B->yb);
        const double t = wabs / d;
        b += lm[i] * pow(t, F->order) / (d * (1.0 - t));
    }
    for (int k = 0; k < B->nacc; ++k) {
        const double mass = B->acc[3 * k], dabs = B->acc[3 * k + 1], rc = B->acc[3 * k + 2];
        const double x = wabs / dabs, y = rc / dabs;
        double e = pow(x / (1.0 - y), F->order) / (1.0 - x - y);
        double xl = 1.0;
        for (int l = 0; l < F->order; ++l) {
            e += xl * binom_tail(l, F->group_order, y, binom);
            xl *= x;
        }
        b += mass / dabs * e;
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
    if (orc_geometry(P, &G) != 0 || !far_params_ok(F) || !counts || !totals || nstar < 0 ||
        P->ray_mode != ORC_RAYS_LATTICE)
        return -1;
    if (nstar > 0 && (!lx || !ly || !lm)) return -1;
    if (i0 < 0) { i0 = 0; i1 = G.nx; j0 = 0; j1 = G.ny; }
    if (i1 > G.nx) i1 = G.nx;
    if (j1 > G.ny) j1 = G.ny;
    if (i1 < i0 || j1 < j0) return -1;
    lens_tree T;
    double *binom = binom_table();
    if (!binom || tree_build(&T, F, lx, ly, lm, nstar) != 0) {
        free(binom);
        tree_free(&T);
        return -1;
    }
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
        if (far_block_build(F, &G, &T, binom, lx, ly, lm, nstar, i0, j0, BX, BY, &B) != 0) {
            err += 1;
            continue;
        }
        const double bb = far_bound(&B, F, binom, lx, ly, lm, B.rho);
        if (bb > bmax) bmax = bb;
        const int64_t ie = i0 + (BX + 1) * bw < i1 ? i0 + (BX + 1) * bw : i1;
        const int64_t je = j0 + (BY + 1) * bh < j1 ? j0 + (BY + 1) * bh : j1;
        for (int64_t j = j0 + BY * bh; j < je; ++j) {
            for (int64_t i = i0 + BX * bw; i < ie; ++i) {
                double x1, x2, a1 = NAN, a2 = NAN;
                ray_position(P, &G, i, j, &x1, &x2);
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
    tree_free(&T);
    free(binom);
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
        !bound || i0 < 0 || j0 < 0 || P->ray_mode != ORC_RAYS_LATTICE)
        return -1;
    lens_tree T;
    double *binom = binom_table();
    if (!binom || tree_build(&T, F, lx, ly, lm, nstar) != 0) {
        free(binom);
        tree_free(&T);
        return -1;
    }
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
        if (far_block_build(F, &G, &T, binom, lx, ly, lm, nstar, i0, j0, (ray_i[k] - i0) / bw, (ray_j[k] - j0) / bh,
                            &B) != 0) {
            err += 1;
            continue;
        }
        double x1, x2, a1 = NAN, a2 = NAN;
        ray_position(P, &G, ray_i[k], ray_j[k], &x1, &x2);
        const int on_lens = far_deflection(&B, F, lx, ly, lm, x1, x2, &a1, &a2);
        pixel[k] = source_pixel(P, &G, x1, x2, a1, a2, on_lens, alpha + 2 * k, ysrc + 2 * k);
        bound[k] = far_bound(&B, F, binom, lx, ly, lm, hypot(x1 - B.xb, x2 - B.yb));
        far_block_free(&B);
    }
    tree_free(&T);
    free(binom);
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
