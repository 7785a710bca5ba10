/*
 * mm.h -- C ABI of the GB300 (sm_103a) microlensing magnification-map library.
 *
 * The library computes magnification maps by direct inverse ray-shooting:
 * every ray of a regular image-plane grid is deflected by all N* point
 * lenses, the smooth-matter and shear terms of the lens equation are added,
 * and the ray is counted into the source-plane pixel where it lands.
 *
 *   Lens equation (Sect. 2, Eq. sigma):
 *     y = diag(1 - gamma, 1 + gamma) x - sigma_c x - sum_i m_i (x - x_i) / |x - x_i|^2
 *     sigma = sigma_c + sigma_*, smooth fraction s = sigma_c / sigma (Sect. 3.1).
 *   Estimator (Sect. 2): mu_ij = N_ij / N_rays, N_rays = mean rays per pixel
 *     without lensing.
 *   Number of lenses (Sect. 2, Eq. nstar): N* = sigma_* A / (pi <M>), A = pi R^2.
 *   Shooting grid (Sect. 3.2.2, Eq. square): L_pm = L / (1 - sigma -+ gamma).
 *
 * Conventions for every entry point:
 *   - Returns MM_OK (0) or a negative MM_E* code; no exception or signal
 *     crosses the ABI; mm_strerror() names the code, mm_last_error() gives
 *     a message for the last failure on the calling thread.
 *   - The caller owns every host buffer it passes; the library never keeps a
 *     pointer to one after the call returns and never frees one.
 *   - The library owns every device object behind an opaque handle
 *     (mm_lenses, mm_map, mm_req) until the matching mm_release_* call or
 *     mm_destroy. Handles are never reused within a context.
 *   - One context is driven from one host thread, except mm_poll, which may
 *     be called from any thread.
 *   - Every kernel runs on the context's CUDA stream (given to mm_init).
 *
 * Geometry readings (where the paper is silent): the shot rectangle is
 * `shoot_margin` times (L/|1-sigma-gamma|, L/|1-sigma+gamma|), centred on
 * the origin; rays form a square lattice of spacing Delta = p / sqrt(N_rays)
 * (p = L / N_side), nx = ceil(W / Delta), ny = ceil(H / Delta), ray (i, j)
 * at ((i + 1/2 - nx/2) Delta, (j + 1/2 - ny/2) Delta); pixel
 * (I, J) = (floor((y1 + L/2)/p), floor((y2 + L/2)/p)), stored at
 * counts[J * N_side + I]; a ray outside [0, N_side)^2, non-finite, or
 * exactly on a lens is counted as "out".
 */
#ifndef MM_H
#define MM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define MM_OK          0
#define MM_EINVAL     -1   /* malformed argument or ill-posed map */
#define MM_ENOMEM     -2   /* over the context's HBM budget, or device allocation failed */
#define MM_EBUSY      -3   /* request queue full */
#define MM_ENOTFOUND  -4   /* unknown or released handle */
#define MM_ETIMEDOUT  -5   /* mm_wait ran out of time (the request is still live) */
#define MM_EDEVICE    -6   /* CUDA error; the context should be destroyed */
#define MM_EAGAIN     -7   /* request not finished yet */
#define MM_ECANCELED  -8   /* request cancelled before it ran */

/* ---- enums ------------------------------------------------------------ */
#define MM_FP32C  0   /* FP32 deflection sum, tile-relative coordinates, compensated
                         accumulation, FP64 near-lens terms, float-float epilogue */
#define MM_FP64   1   /* plain FP64 everywhere */
#define MM_FAR32  2   /* far-field approximation, the tree code's idea (Sect. 2.1, Eq.
                         hierarchical) on blocks of rays: the ray lattice is cut into
                         blocks of far_block x far_block tiles (64 x 32 rays each);
                         lenses within rho / far_ratio of a block's centre (rho: the
                         block's half-diagonal) are summed exactly for each of its rays
                         (FP32 with FP64 terms near the tile, as MM_FP32C); the others
                         enter far_order terms of the series of sum m / (z - z_i) about
                         the centre. Per-ray truncation error <= sum over far lenses of
                         m t^P / (|d| (1 - t)), t = |z - z_B| / |d| < far_ratio, d the
                         lens offset from the centre; its largest value over the map's
                         blocks is mm_stats.far_bound. Cost per ray: P complex FMAs plus
                         the near lenses, instead of N* interactions. */

#define MM_MASS_UNIT       0   /* m_i = 1 */
#define MM_MASS_LOGNORMAL  1   /* m_i = exp(mass_mu + mass_s z), z ~ N(0, 1) */

typedef struct mm_ctx mm_ctx;
typedef uint64_t mm_lenses;   /* 0 is never a valid handle */
typedef uint64_t mm_map;
typedef uint64_t mm_req;

/* Map request, in the paper's terms (Sect. 2 and 3.1). */
typedef struct {
    double   sigma;          /* total convergence sigma (Eq. sigma) */
    double   gamma;          /* external shear gamma */
    double   smooth_frac;    /* s = sigma_c / sigma, in [0, 1] */
    double   side_re;        /* source-plane side L in Einstein radii of a unit mass, > 0 */
    int32_t  npix_side;      /* N_side, 1 .. 32768; N_pix = N_side^2 */
    double   nrays_per_pix;  /* N_rays > 0: mean rays per pixel without lensing */
    double   shoot_margin;   /* shot rectangle per side / mapped-back source side; <= 0 means 1.5 */
    int32_t  precision;      /* MM_FP32C or MM_FP64 */
    int64_t  nstar;          /* N*; < 0: derived (Eq. nstar with the disc rule below) */
    double   disc_radius;    /* lens-disc radius R; <= 0: derived */
    int32_t  mass_model;     /* MM_MASS_UNIT or MM_MASS_LOGNORMAL */
    double   mass_mu;        /* lognormal mu */
    double   mass_s;         /* lognormal s */
    uint64_t seed;           /* lens-field seed (SplitMix64 streams) */
    int64_t  ray_rect[4];    /* [i0, i1, j0, j1) sub-rectangle of the global ray grid, or
                                all -1 for the whole grid (tests and windowed runs) */
    int32_t  far_order;      /* MM_FAR32: series terms P, 1 .. 32 (default 10) */
    double   far_ratio;      /* MM_FAR32: near ratio q, 0 < q <= 0.9 (default 0.15) */
    int32_t  far_block;      /* MM_FAR32: block side in ray tiles, 1 .. 64, or 0 (default): the
                                side that minimises a cost model of block preparation
                                (blocks x N* x P) against near-lens work (rays x near lenses
                                per block), from the whole ray grid, the lens count and the
                                largest lens distance from the origin.
                                Blocks are counted from the origin of the shot rectangle */
    int32_t  far_group_order;/* MM_FAR32: grouped far lenses (the tree code's cells, Sect. 2.1):
                                K multipole moments per cell of a lens quadtree, 1 .. 32 (needs
                                far_order <= 16); 0: every far lens enters its block's series
                                alone; -1 (default): 24 when a cost model of the block setup finds
                                grouping faster (in practice from about 1e6 lenses on), else 0. The
                                automatic block side (far_block = 0) comes from the same model.
                                The tree: R0 = the smallest power of two above every
                                |x_i|, |y_i|; level L cuts [-R0, R0)^2 into cells of side
                                2 R0 / 2^L; a cell with more than far_group_leaf lenses (below
                                level 16) splits into its four quadrants. For block B a cell C
                                (centre z_C, half-diagonal r_C, D = z_C - z_B) is grouped when
                                |D| - r_C >= rho / far_ratio and rho + r_C <= far_group_theta |D|;
                                its moments a_k = sum m_i (z_i - z_C)^k then add
                                -sum_{k<K} (-1)^k C(l+k, k) a_k / D^(l+k+1) to c_l, and its lenses
                                are not examined one by one. The near lenses are the same as
                                without grouping. A grouped cell adds (M_C / |D|) E(x, y) to the
                                bound, x = rho / |D|, y = r_C / |D|,
                                E = (x / (1 - y))^P / (1 - x - y) + sum_{l<P} x^l sum_{k>=K} C(l+k, k) y^k */
    double   far_group_theta;/* MM_FAR32 grouping: separation theta, 0 < theta <= 0.9 (default 0.3) */
    int32_t  far_group_leaf; /* MM_FAR32 grouping: most lenses of a leaf cell, 1 .. 2^20 (default 64) */
    int32_t  ray_mode;       /* MM_RAYS_LATTICE (0, default): ray (i, j) at the centre of lattice
                                cell (i, j), the tree code's regular grid (Sect. 3.1).
                                MM_RAYS_RANDOM (1): at a pseudo-random position, as the paper's GPU
                                code shoots its rays (Sect. 2.3, step 2), so that a pixel receives
                                N_rays rays on average only (Sect. 3.1). The same nx * ny rays are
                                shot; ray (i, j) is uniform in the 64 x 32-cell tile of the lattice
                                that holds cell (i, j): with q = j nx + i, u1 and u2 the top 18 bits
                                of outputs 2q + 1 and 2q + 2 of SplitMix64(ray_seed) (output k of
                                the generator seeded with s is mix(s + k 0x9E3779B97F4A7C15)), as
                                fractions in [0, 1), Ti = floor(i / 64), Tj = floor(j / 32),
                                wi = min(64, nx - 64 Ti), wj = min(32, ny - 32 Tj):
                                x1 = (64 Ti + u1 wi - nx/2) Delta, x2 = (32 Tj + u2 wj - ny/2) Delta.
                                For MM_FP32C and MM_FP64 through mm_shoot, mm_shoot_batch,
                                mm_shoot_into and mm_debug_deflect; ray_rect must start on the
                                64 x 32-ray tile grid (i0 % 64 == 0, j0 % 32 == 0). MM_FAR32,
                                mm_submit and mm_shoot_noalloc take the lattice only (MM_EINVAL). */
    uint64_t ray_seed;       /* MM_RAYS_RANDOM: seed of the ray positions (default 1) */
} mm_params;

#define MM_RAYS_LATTICE 0
#define MM_RAYS_RANDOM  1

/* Lens-field derivation used by mm_create_lenses when nstar < 0 or
 * disc_radius <= 0 (reading of Sect. 2, after Eq. nstar: lenses fill a
 * circle wider than the mapped-back source region):
 *   R  = (shoot_margin / 2) * hypot(L/|1-sigma-gamma|, L/|1-sigma+gamma|) + 2,
 *   N* = round(sigma_* R^2 / <M>),   sigma_* = (1 - s) sigma,
 * and, when only N* is given, R = sqrt(N* <M> / sigma_*).
 * <M> = 1 (unit) or exp(mass_mu + mass_s^2 / 2) (lognormal). */

typedef struct {
    uint64_t rays_shot;     /* rays of the (sub-)grid shot: nx * ny, or the rectangle's area */
    uint64_t rays_in;       /* rays counted into the map */
    uint64_t rays_out;      /* rays outside the map, non-finite or on a lens */
    uint64_t interactions;  /* rays_shot * N* */
    uint64_t nx, ny;        /* global ray-grid size */
    int64_t  nstar;
    double   seconds;       /* device time of the map's shoot, CUDA events (0 if unknown) */
    double   mu_mean;       /* rays_in / (N_side^2 N_rays) */
    int32_t  lens_splits;   /* lens segments per ray tile: maps with few tiles (< 2048) and many
                               lenses (> 1024) spread each tile's lens sum over several CTAs and
                               combine the segments' float-float sums in segment order */
    double   far_bound;     /* MM_FAR32: largest truncation bound of any ray (Einstein radii,
                               evaluated at the block radius); 0 for the exact precisions */
    int32_t  far_block;     /* MM_FAR32: the block side (tiles) used; 0 for the exact precisions */
    int32_t  far_group;     /* MM_FAR32: the multipole order K of grouped cells (0: no grouping) */
} mm_stats;

typedef struct {
    double  pix;        /* p = L / N_side */
    double  delta;      /* lattice spacing p / sqrt(N_rays) */
    double  width;      /* shot rectangle W */
    double  height;     /* shot rectangle H */
    int64_t nx, ny;     /* global ray-grid size */
    int64_t nstar;      /* N* after derivation */
    double  disc_radius;
    double  mu_theory;  /* 1 / ((1 - sigma)^2 - gamma^2), Eq. mutheory */
    int32_t far_block;  /* MM_FAR32: the block side in tiles for these parameters (the automatic
                           choice when far_block = 0, for the N* and disc radius above; a map
                           shot with another lens set reports its own in mm_stats) */
    int32_t far_group;  /* MM_FAR32: the multipole order K of grouped cells for these parameters
                           (the automatic choice when far_group_order = -1), 0: no grouping */
} mm_geometry;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`. hbm_budget_bytes caps the device
 * memory the context may hold (0: 90 % of the free memory at init).
 * cuda_stream is a cudaStream_t (for example torch.cuda.current_stream()
 * .cuda_stream) or NULL for a stream the library creates. *out receives the
 * context. Errors: MM_EINVAL (out NULL, bad device), MM_EDEVICE. */
int mm_init(mm_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream);

/* Wait for all work, release every object and the context. NULL is a no-op. */
int mm_destroy(mm_ctx *ctx);

/* ---- parameters and geometry (host only, no device work) -------------- */

/* Fill *p with the defaults: margin 1.5, MM_FP32C, derived N* and R, unit
 * masses, seed 1, whole grid. Physical fields are zero and must be set. */
int mm_params_default(mm_params *p);

/* Validate *p and compute its geometry and derived lens-field size.
 * Errors: MM_EINVAL (|1-sigma-+gamma| < 1e-3, side <= 0, N_side outside
 * 1..32768, N_rays <= 0, smooth_frac outside [0, 1], bad enums, ray_rect
 * outside the grid). */
int mm_geometry_of(const mm_params *p, mm_geometry *g);

/* ---- lens sets ---------------------------------------------------------- */

/* Generate a seeded lens field on the host in FP64 (N* and R per the rule
 * above; positions uniform in the disc by rejection sampling from the
 * SplitMix64 stream seeded from p->seed; unit or lognormal masses), copy it
 * to the device once, and build the FP32 tile copies there. Errors:
 * MM_EINVAL, MM_ENOMEM (over budget), MM_EDEVICE. */
int mm_create_lenses(mm_ctx *ctx, const mm_params *p, mm_lenses *out);

/* The same from caller arrays x[n], y[n], m[n] (FP64, Einstein radii and
 * unit masses); n may be 0. The arrays are copied before return. */
int mm_create_lenses_from(mm_ctx *ctx, const double *x, const double *y, const double *m,
                          int64_t n, mm_lenses *out);

/* Copy a lens set back to caller arrays of n entries each (n must equal the
 * set's size; any pointer may be NULL to skip that array). */
int mm_lenses_fetch(mm_ctx *ctx, mm_lenses h, double *x, double *y, double *m, int64_t n);

/* Number of lenses in a set. */
int mm_lenses_count(mm_ctx *ctx, mm_lenses h, int64_t *n);

int mm_release_lenses(mm_ctx *ctx, mm_lenses h);

/* ---- synchronous shooting ---------------------------------------------- */

/* Shoot one map (Sect. 2, inverse ray-shooting) with lens set `lenses` (0:
 * generate one from *p, owned by the map) and return its handle when the
 * map is complete on the device. The uint32 counts stay in HBM until
 * mm_map_fetch / mm_release_map. Errors: MM_EINVAL, MM_ENOTFOUND,
 * MM_ENOMEM, MM_EDEVICE. */
int mm_shoot(mm_ctx *ctx, mm_lenses lenses, const mm_params *p, mm_map *out);

/* Shoot n maps in ONE persistent launch (maps of different shapes, N* and
 * precision=MM_FP32C share the launch; work is split into ray tiles that the
 * CTAs take from a device counter). lenses[k] may be 0 (generated from
 * params[k]). Each map's result is bit-identical to shooting it alone.
 * maps_out[n] receives the handles. */
int mm_shoot_batch(mm_ctx *ctx, int32_t n, const mm_lenses *lenses, const mm_params *params,
                   mm_map *maps_out);

/* Shoot the rays of p's ray_rect (the image-plane lattice of Sect. 2, in part)
 * into an existing map, whose counts and totals add up: a map can be shot in
 * parts, for example band by band, and resumed after an interruption from the
 * first part not yet shot. p must equal the map's parameters except ray_rect;
 * lenses (0: the map's own lens set) must have the map's lens count. Each
 * part's tiles sum their lenses as mm_shoot over the whole ray grid does (the
 * map's kernel variant, the whole grid's lens split) and integer counts
 * commute, so parts whose ray_rect starts on the 64 x 32-ray tile grid
 * (i0 % 64 == 0, j0 % 32 == 0), shot into a map made with an empty ray_rect
 * and covering the grid once, give that one-shot map bit for bit. Blocks until
 * the part is shot. Errors: MM_EINVAL, MM_ENOTFOUND, MM_ENOMEM, MM_EDEVICE. */
int mm_shoot_into(mm_ctx *ctx, mm_lenses lenses, const mm_params *p, mm_map map);

/* Recreate a map from a checkpoint: host_counts[n_elems] and *st as
 * mm_map_fetch returned them (rays_shot, rays_in, rays_out, nx, ny, nstar,
 * seconds and far_bound are read). p must hold the map's parameters (ray_rect is ignored);
 * lenses (0: generated from p, as mm_shoot does) must have st->nstar lenses.
 * The new map continues with mm_shoot_into; the rays already shot are the
 * caller's record. Copies the host data before it returns. Errors: MM_EINVAL
 * (sizes, or counts that do not sum to rays_in, or rays_in + rays_out !=
 * rays_shot, or a geometry or lens count other than the checkpoint's),
 * MM_ENOTFOUND, MM_ENOMEM, MM_EDEVICE. */
int mm_map_restore(mm_ctx *ctx, mm_lenses lenses, const mm_params *p, const uint32_t *host_counts, size_t n_elems,
                   const mm_stats *st, mm_map *out);

/* Copy a map to host_counts[n_elems] (n_elems must equal N_side^2; may be
 * NULL to fetch only the stats) and fill *st (may be NULL). Blocks until
 * the map is complete. */
int mm_map_fetch(mm_ctx *ctx, mm_map map, uint32_t *host_counts, size_t n_elems, mm_stats *st);

/* Normalised map on the device, copied to host_out[n_elems] (n_elems = N_side^2,
 * row-major, FP32):
 *   MM_MAP_MU       mu_ij = N_ij / N_rays (Sect. 2, the inverse ray-shooting estimator);
 *   MM_MAP_DELTA_M  Delta m_ij = -2.5 log10(max(N_ij, 1) / N_rays) (Eq. deltam), an empty
 *                   pixel clamped to one ray (the paper gives no value for mu = 0).
 * *n_empty (may be NULL) receives the number of pixels with N_ij = 0 (the clamped ones).
 * FP32 arithmetic: mu within 2e-7 relative, Delta m within 1e-5 mag of the FP64 values.
 * Blocks until the map is complete. Errors: MM_EINVAL (kind, NULL buffer or wrong
 * n_elems), MM_ENOTFOUND, MM_ENOMEM, MM_EDEVICE. */
#define MM_MAP_MU       0
#define MM_MAP_DELTA_M  1
int mm_map_fetch_mu(mm_ctx *ctx, mm_map map, int32_t kind, float *host_out, size_t n_elems, int64_t *n_empty);

/* Device address of a map's uint32 counts (N_side^2, row-major), valid until
 * mm_release_map; for zero-copy use on the context's stream. */
int mm_map_device_ptr(mm_ctx *ctx, mm_map map, void **dptr, size_t *n_elems);

int mm_release_map(mm_ctx *ctx, mm_map map);

/* ---- serving: continuous batching ----------------------------------------
 * A request is admitted when a slot is free and its footprint (lens set +
 * map + tile bookkeeping) fits the HBM budget; admitted requests are shot
 * in waves: each wave is one persistent launch (replayed from a captured
 * CUDA graph) over ray tiles of every admitted map, so maps that arrive
 * while others run join at the next wave and their work overlaps on the
 * device. Results are bit-identical to mm_shoot of the same map. */

/* Enqueue a map request; never blocks. lenses may be 0 (the library
 * generates the field from *p when the request is admitted). Errors:
 * MM_EINVAL, MM_EBUSY (queue full), MM_ENOMEM (footprint can never fit). */
int mm_submit(mm_ctx *ctx, mm_lenses lenses, const mm_params *p, mm_req *out);

/* Non-blocking: *done = 1 and *map_out set when the request finished
 * (the map is then owned by the caller as from mm_shoot), 0 otherwise.
 * Returns the request's error code if it failed. */
int mm_poll(mm_ctx *ctx, mm_req req, int *done, mm_map *map_out);

/* Block until the request finishes or timeout_ns elapses (< 0: forever).
 * Errors: MM_ETIMEDOUT (still running), or the request's own error. */
int mm_wait(mm_ctx *ctx, mm_req req, int64_t timeout_ns, mm_map *map_out);

/* Cancel a request. A queued request ends at once; an admitted one stops before its
 * next work item is scheduled (work already on the GPU finishes first, and the map
 * is dropped); either way it then reports MM_ECANCELED. MM_EBUSY if the request has
 * finished or all of its work is already on the GPU (it will complete normally). */
int mm_cancel(mm_ctx *ctx, mm_req req);

/* Serving counters since the context's server started (all zero before the first
 * mm_submit or mm_serve_config). */
typedef struct {
    uint64_t waves;         /* waves completed */
    uint64_t items;         /* work items (ray tiles, or far-field block rows) they shot */
    double   interactions;  /* ray-lens interactions of those items: each item's share of its
                               map's rays x N* (for far-field maps, the exact method's count) */
    uint64_t completed, cancelled, failed;   /* requests ended each way */
    int32_t  queued;        /* requests waiting for admission now */
    int32_t  preparing;     /* admitted, lens field and map being prepared */
    int32_t  active;        /* admitted and prepared, being shot */
} mm_serve_stats_t;
int mm_serve_stats(mm_ctx *ctx, mm_serve_stats_t *out);

/* Latency of a finished request: submit -> admit -> done, seconds (host clock). */
int mm_req_times(mm_ctx *ctx, mm_req req, double *t_queue, double *t_total);

/* Serving limits: max concurrently admitted maps (default 64), max queued
 * requests (65536), and the target device time of one wave in milliseconds
 * (default 12; 0 keeps the current value of any argument). A request completes
 * about two waves after it joins one, so the wave length sets the latency floor;
 * waves below ~8 ms lose throughput to launch overhead. */
int mm_serve_config(mm_ctx *ctx, int32_t max_active, int32_t max_queued, double wave_ms);

/* How a wave's work budget (about wave_ms of device time) is divided between
 * the admitted maps: the share priority_share (0..1, default 0.8) goes to the
 * maps in increasing order of remaining work (shortest remaining work first),
 * the rest evenly to all of them (processor sharing); every map with work
 * left gets at least one work item per wave, so none starves. 0 is plain
 * processor sharing. Admission from the queue stays first come, first served.
 * Applies from the next wave. Errors: MM_EINVAL (share outside [0, 1]). */
int mm_serve_priority(mm_ctx *ctx, double priority_share);

/* The division above as a pure host function (no context, no GPU), for
 * inspection and tests. n maps with left[k] work items remaining, each worth
 * cost[k] > 0 interactions (or their device-time equivalent); budget > 0 in
 * the same unit. Writes take[k], the items of map k in the wave: a
 * priority_share of the budget to the maps in increasing order of
 * left[k] * cost[k] (ties by index), each taking up to ceil(rest / cost[k])
 * items while budget remains, then floor((1 - priority_share) budget /
 * (n cost[k])) more items, at least one, per map; take[k] <= left[k]. The
 * budget is doubled (up to 64 times) until the wave holds at least
 * min(min_items, sum of left) items. Errors: MM_EINVAL. */
int mm_serve_plan(const uint64_t *left, const double *cost, int32_t n, double budget, double priority_share,
                  uint64_t min_items, uint64_t *take);

/* ---- map statistics (Sect. 3.1, Eq. deltam) --------------------------------
 * The paper compares maps by the RMS difference of Delta m = -2.5 log10(mu)
 * (mu = N / N_rays per pixel) and by a two-sample Kolmogorov-Smirnov test on the
 * Delta m distributions ("excellent agreement": RMS < 0.2 mag and K-S probability
 * > 99.7 %). Readings: the RMS runs over pixels where both maps count at least
 * one ray; empty pixels enter the K-S test with Delta m = +infinity; the K-S
 * probability is the asymptotic Kolmogorov distribution at
 * (sqrt(n_e) + 0.12 + 0.11/sqrt(n_e)) D, n_e = n_a n_b / (n_a + n_b). */
typedef struct {
    double  rms_dm;      /* RMS of Delta m_a - Delta m_b over pixels counted in both maps, mag */
    int64_t n_rms;       /* pixels in the RMS */
    int64_t zero_a;      /* empty pixels of map a */
    int64_t zero_b;      /* empty pixels of map b */
    double  ks_d;        /* K-S statistic of the Delta m distributions (exact) */
    double  ks_p;        /* asymptotic K-S probability (null hypothesis not rejected) */
    double  mean_mu_a;   /* mean magnification of each map */
    double  mean_mu_b;
} mm_compare;

/* Compare two maps of the same N_side on the device (each map's own N_rays sets
 * its mu). Waits for both maps. Errors: MM_EINVAL (different N_side),
 * MM_ENOTFOUND, MM_EDEVICE. */
int mm_map_compare(mm_ctx *ctx, mm_map a, mm_map b, mm_compare *out);

/* ---- extended sources (Sect. 1) --------------------------------------------
 * A finite source's magnification at each position: the point-source map
 * convolved with its brightness profile. mu = N / N_rays per pixel; the profile is discretised on the pixel
 * grid and normalised to unit sum:
 *   MM_PROFILE_GAUSSIAN  w(i, j) = g(i) g(j), g(k) = exp(-(k p)^2 / (2 size^2)),
 *                        |k| <= ceil(4 size / p) (square support, separable);
 *   MM_PROFILE_DISC      w(i, j) = 1 where (i^2 + j^2) p^2 <= size^2 (uniform disc).
 * Output pixels whose profile support leaves the map are NaN. */
#define MM_PROFILE_GAUSSIAN 0
#define MM_PROFILE_DISC     1

/* Convolved magnification map into host_mu[n_elems] (n_elems = N_side^2, row-major,
 * float). size_re: Gaussian sigma or disc radius in Einstein radii. Errors:
 * MM_EINVAL (bad profile or size, profile wider than the map, wrong n_elems),
 * MM_ENOTFOUND, MM_EDEVICE. */
int mm_map_convolve(mm_ctx *ctx, mm_map map, int32_t profile, double size_re, float *host_mu, size_t n_elems);

/* Light curve of an extended source moving on a straight track from (y1_start,
 * y2_start) to (y1_end, y2_end) (source-plane Einstein radii, origin at the map
 * centre): n_points samples, evenly spaced including both ends, of the convolved
 * map, bilinearly interpolated between pixel centres (-L/2 + (I + 1/2) p);
 * host_mu[k] is NaN where a sample needs a pixel without value. When it is less
 * work, only the four pixels around each sample are convolved (one CTA per
 * sample) instead of the whole map; either way every pixel, and so every sample,
 * equals what sampling mm_map_convolve's map gives, bit for bit. Errors:
 * MM_EINVAL (bad profile or size, profile wider than the map, n_points <= 0,
 * NULL host_mu), MM_ENOTFOUND, MM_ENOMEM, MM_EDEVICE. */
int mm_map_lightcurve(mm_ctx *ctx, mm_map map, int32_t profile, double size_re, double y1_start, double y2_start,
                      double y1_end, double y2_end, int64_t n_points, double *host_mu);

/* ---- tuning and inspection ------------------------------------------------ */

/* Autotune for maps like *p: time every thread layout x tile variant of the
 * FP32 kernel on a window of about 600 tiles of such a map, keep the fastest
 * layout for the context and record the fastest variant for maps of p's class
 * (unit vs lognormal masses, N* bucket by powers of two); *variant receives it.
 * Layouts give bit-identical maps; variants differ only in rounding. */
int mm_autotune(mm_ctx *ctx, const mm_params *p, int32_t *variant);

/* Force a tile variant for subsequent FP32 shoots (-1: use the tuned table,
 * else the default: variant 0 for unit masses, 2 for lens sets with masses).
 * A variant fixes the share of lens pairs whose two reciprocals come from one
 * reciprocal of their product, and the compensated-fold interval. */
int mm_set_variant(mm_ctx *ctx, int32_t variant);

/* Number of FP32 tile variants and a description of one. */
int mm_variant_count(void);
const char *mm_variant_name(int32_t variant);

/* Set or read the FP32 thread layout of the context (how a 64 x 32-ray tile is
 * split over threads); MM_EBUSY once serving has started. */
int mm_set_layout(mm_ctx *ctx, int32_t layout);
int mm_get_layout(mm_ctx *ctx, int32_t *layout);
int mm_layout_count(void);
const char *mm_layout_name(int32_t layout);

/* Per-ray deflection through the same kernel code as the map: for rays
 * (ray_i[k], ray_j[k]) of the global grid, alpha_out[2k..2k+1] receives the
 * star deflection sum_i m_i (x - x_i)/|x - x_i|^2 (Eq. sigma) and pixel_out[k]
 * the flat pixel index the map kernel would count the ray into (-1: out).
 * Any output pointer may be NULL. */
int mm_debug_deflect(mm_ctx *ctx, mm_lenses lenses, const mm_params *p,
                     const int64_t *ray_i, const int64_t *ray_j, int64_t n,
                     double *alpha_out, int64_t *pixel_out);

/* Test hook for the device's own time limits: arm a one-shot failure that the
 * next call of the named kind meets on the device, so that a test can check the
 * error path without faulting the GPU.
 *   MM_INJECT_COMPARE_NO_COPY  the next mm_map_compare issues none of its bulk
 *     copies into shared memory: its waits for them give up after their limit
 *     (about one second of SM clocks), the call returns MM_EDEVICE, and the
 *     context stays usable.
 *   MM_INJECT_DISC_NO_COPY  the next disc convolution (mm_map_convolve or
 *     mm_map_lightcurve with MM_PROFILE_DISC, radius up to 15 pixels) announces
 *     but issues none of the bulk copies that stage its interior tiles: those
 *     waits give up after their limit, the call returns MM_EDEVICE, and the
 *     context stays usable.
 * An armed failure stays armed until a call of its kind takes it.
 * MM_INJECT_NONE disarms. Errors: MM_EINVAL (null context, unknown kind). */
#define MM_INJECT_NONE             0
#define MM_INJECT_COMPARE_NO_COPY  1
#define MM_INJECT_DISC_NO_COPY     2
int mm_debug_inject(mm_ctx *ctx, int32_t kind);

/* ---- shooting without allocation --------------------------------------------
 * The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory, such as code running under another runtime or
 * framework that owns the GPU's memory and accounts for every byte, or a tight
 * loop that cannot afford the device-wide synchronisation of cudaMalloc and
 * cudaFree. It shoots one map with the FP32 kernel (thread layout and tile
 * variant of a fresh context) and allocates nothing: no context is needed, and
 * the kernel's scratch (FP32 lens tile copies, launch header, map descriptor,
 * work counter) lives in one fixed __device__ array of about 2.6 MB that every
 * GPU which loads the library holds until the process exits. Each ray tile sums
 * all its lenses in one CTA: for maps that mm_shoot does not split over lens
 * segments (2048 tiles or more, or 1024 lenses or fewer) the counts equal
 * mm_shoot's on a fresh context bit for bit; maps that mm_shoot splits may
 * differ from it by rounding at pixel edges, within the FP32 path's tolerances.
 *   x, y, m   device arrays of nstar FP64 lens coordinates and masses, owned by
 *             the caller; m is not read (may be NULL) when p->mass_model is
 *             MM_MASS_UNIT. p->nstar and p->disc_radius are ignored.
 *   nstar     0 .. 131072 (the scratch capacity); larger values return MM_EINVAL.
 *   p         map parameters; p->precision must be MM_FP32C.
 *   counts    device array of N_side^2 uint32 (row-major map), owned by the
 *             caller; zeroed by the call.
 *   totals    device array of 2 uint64 {rays in, rays out}; zeroed by the call.
 *   cuda_stream  the stream to run on (NULL: the default stream).
 * Runs on the current CUDA device; all pointers must belong to it. The call
 * returns once the work is enqueued; the outputs are complete when the stream
 * reaches it. The first call on a device looks up the scratch's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture. The address is kept for the rest of the process and is
 * valid for the device's primary context: do not call this entry point on a
 * device after cudaDeviceReset has destroyed that context. Every call shares the
 * one scratch array, which keeps the last call's contents: calls whose work
 * overlaps on the GPU (other streams, other threads) race and give wrong maps --
 * serialise them. Errors: MM_EINVAL, MM_EDEVICE. */
int mm_shoot_noalloc(const double *x, const double *y, const double *m, int64_t nstar, const mm_params *p,
                     uint32_t *counts, uint64_t *totals, void *cuda_stream);

/* Device time (ms) of the kernels of the most recent shoot, batch, debug,
 * convolution or light-curve call, measured with CUDA events on the context's
 * stream around them, and the number of kernels in that time. */
int mm_last_kernel_ms(mm_ctx *ctx, double *ms, int32_t *launches);

const char *mm_strerror(int code);
const char *mm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MM_H */
