/* mm_oracle.h -- plain FP64 CPU oracle (test infrastructure only; see mm_oracle.c). */
#ifndef MM_ORACLE_H
#define MM_ORACLE_H
#include <stdint.h>

typedef struct {
    double sigma;        /* total convergence sigma = sigma_c + sigma_* (Eq. sigma) */
    double gamma;        /* external shear */
    double smooth_frac;  /* s = sigma_c / sigma */
    double side;         /* source-plane side L, Einstein radii */
    int32_t npix_side;   /* N_side; the map has N_side^2 pixels */
    double nrays;        /* N_rays: mean rays per pixel without lensing */
    double margin;       /* shot rectangle = margin x (L/|a|, L/|b|) per side */
    int32_t ray_mode;    /* ORC_RAYS_LATTICE (0): ray (i, j) at the centre of lattice cell (i, j);
                            ORC_RAYS_RANDOM (1): at a pseudo-random position in the 64 x 32-cell
                            tile of the lattice that holds cell (i, j) (see ray_position) */
    uint64_t ray_seed;   /* seed of the random positions (ORC_RAYS_RANDOM) */
} orc_params;

#define ORC_RAYS_LATTICE 0
#define ORC_RAYS_RANDOM  1

typedef struct {
    double pix, delta, width, height;
    int64_t nx, ny;
} orc_geometry_t;

int orc_geometry(const orc_params *P, orc_geometry_t *G);

/* Map over the ray sub-rectangle [i0,i1) x [j0,j1) of the global grid, taking every
 * `stride`-th ray in each direction (i0 < 0: the whole grid). counts has N_side^2
 * entries; totals = {shot, in, out}. */
int orc_map(const orc_params *P, const double *lx, const double *ly, const double *lm, int64_t nstar,
            int64_t i0, int64_t i1, int64_t j0, int64_t j1, int64_t stride,
            uint32_t *counts, uint64_t totals[3], int nthreads);

/* Per-ray deflection alpha[2k..2k+1], source position ysrc[2k..2k+1] and flat pixel
 * (or -1) of rays (ray_i[k], ray_j[k]). */
int orc_rays(const orc_params *P, const double *lx, const double *ly, const double *lm, int64_t nstar,
             const int64_t *ray_i, const int64_t *ray_j, int64_t n,
             double *alpha, double *ysrc, int64_t *pixel, int nthreads);

/* Far-field approximation on blocks of rays (see mm_oracle.c): series order P,
 * near ratio q (a lens is summed exactly iff |d| < rho / q) and the block side
 * in 64 x 32-ray tiles; blocks are counted from the shot rectangle's origin. */
typedef struct {
    int32_t order;        /* P >= 1 */
    double ratio;         /* q in (0, 1) */
    int32_t block_tiles;  /* bt >= 1: a block is 64 bt x 32 bt rays */
    int32_t group_order;  /* K: multipole terms of a lens cell; 0: no grouping (every far lens alone) */
    double group_theta;   /* theta in (0, 1): a cell is grouped when (rho + r_C) <= theta |z_C - z_B| */
    int32_t group_leaf;   /* a cell of the lens tree with more lenses than this is split (>= 1) */
} orc_far_params;

/* Map of the rectangle [i0,i1) x [j0,j1) (i0 < 0: the whole grid) with the far
 * field of each block replaced by its truncated series; *bound_max = the largest
 * truncation bound of any block (at |w| = rho). */
int orc_far_map(const orc_params *P, const orc_far_params *F, const double *lx, const double *ly, const double *lm,
                int64_t nstar, int64_t i0, int64_t i1, int64_t j0, int64_t j1,
                uint32_t *counts, uint64_t totals[3], double *bound_max, int nthreads);

/* Per-ray far-field deflection, source position, pixel and truncation bound of
 * rays (ray_i[k], ray_j[k]) of a rectangle whose origin is (i0, j0). */
int orc_far_rays(const orc_params *P, const orc_far_params *F, const double *lx, const double *ly, const double *lm,
                 int64_t nstar, int64_t i0, int64_t j0, const int64_t *ray_i, const int64_t *ray_j, int64_t n,
                 double *alpha, double *ysrc, int64_t *pixel, double *bound, int nthreads);

int orc_max_threads(void);
#endif
