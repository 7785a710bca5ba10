// mm_host.cpp -- host runtime of the C ABI: validation and geometry (FP64),
// seeded lens fields, the device arena, object tables and the synchronous,
// batched and debug shooting calls. The serving loop is in mm_serve.cpp.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "mm_ctx.h"

namespace mm {

// ---------------------------------------------------------------- errors ---

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg)
{
    set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) return fail(MM_ENOMEM, std::string(what) + ": " + cudaGetErrorString(e));
    return fail(MM_EDEVICE, std::string(what) + ": " + cudaGetErrorString(e));
}


// ------------------------------------------------ seeded lens field (FP64) ---
// SplitMix64 (Steele, Lea & Flood 2014): output k of a generator seeded with s
// is mix64(s + k * golden_gamma). Positions: rejection sampling from the
// square [-R, R)^2, candidate c using outputs 2c+1, 2c+2; masses: lognormal by
// the Box-Muller cosine branch on outputs 2i+1, 2i+2 of the mass stream.

static constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ULL;

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline double uniform01(uint64_t seed, uint64_t k)
{
    return (double)(mix64(seed + k * kGolden) >> 11) * 0x1.0p-53;
}

static void generate_field(uint64_t seed, long long n, double radius, int mass_model, double mu, double s,
                           std::vector<double> &x, std::vector<double> &y, std::vector<double> &m)
{
    const uint64_t pos_seed = mix64(seed + kGolden);
    const uint64_t mass_seed = mix64(seed + 2 * kGolden);
    x.resize((size_t)n);
    y.resize((size_t)n);
    m.resize((size_t)n);
    long long have = 0;
    for (uint64_t c = 0; have < n; ++c) {
        const double u1 = uniform01(pos_seed, 2 * c + 1);
        const double u2 = uniform01(pos_seed, 2 * c + 2);
        const double px = radius * (2.0 * u1 - 1.0);
        const double py = radius * (2.0 * u2 - 1.0);
        const double rr = px * px;
        const double r2 = rr + py * py;
        if (r2 < radius * radius) {
            x[(size_t)have] = px;
            y[(size_t)have] = py;
            ++have;
        }
    }
    for (long long i = 0; i < n; ++i) {
        if (mass_model == MM_MASS_UNIT) {
            m[(size_t)i] = 1.0;
        } else {
            const double u1 = 1.0 - uniform01(mass_seed, 2 * (uint64_t)i + 1);
            const double u2 = uniform01(mass_seed, 2 * (uint64_t)i + 2);
            const double z = std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
            m[(size_t)i] = std::exp(mu + s * z);
        }
    }
}

// ------------------------------------------------------------- geometry ---

static bool finite(double v) { return std::isfinite(v); }

int compute_geo(const mm_params *p, Geo *g)
{
    if (!p || !g) return fail(MM_EINVAL, "null params");
    if (p->precision != MM_FP32C && p->precision != MM_FP64 && p->precision != MM_FAR32)
        return fail(MM_EINVAL, "precision must be MM_FP32C, MM_FP64 or MM_FAR32");
    if (p->precision == MM_FAR32) {
        if (p->far_order < 1 || p->far_order > kFarMaxOrder) return fail(MM_EINVAL, "far_order must be in 1..32");
        if (!finite(p->far_ratio) || !(p->far_ratio > 0.0) || p->far_ratio > 0.9)
            return fail(MM_EINVAL, "far_ratio must be in (0, 0.9]");
        if (p->far_block < 0 || p->far_block > kFarMaxBlock) return fail(MM_EINVAL, "far_block must be in 0..64");
        if (p->far_group_order < -1 || p->far_group_order > kGroupMaxOrder)
            return fail(MM_EINVAL, "far_group_order must be -1 (automatic), 0 or 1..32");
        if (p->far_group_order > 0 && p->far_order > kGroupMaxSeries)
            return fail(MM_EINVAL, "grouped far lenses need far_order <= 16");
        if (!finite(p->far_group_theta) || !(p->far_group_theta > 0.0) || p->far_group_theta > 0.9)
            return fail(MM_EINVAL, "far_group_theta must be in (0, 0.9]");
        if (p->far_group_leaf < 1 || p->far_group_leaf > (1 << 20)) return fail(MM_EINVAL, "far_group_leaf must be in 1..2^20");
    }
    if (p->mass_model != MM_MASS_UNIT && p->mass_model != MM_MASS_LOGNORMAL) return fail(MM_EINVAL, "bad mass_model");
    if (!finite(p->sigma) || !finite(p->gamma) || p->sigma < 0.0) return fail(MM_EINVAL, "sigma must be finite and >= 0, gamma finite");
    if (!finite(p->side_re) || !(p->side_re > 0.0)) return fail(MM_EINVAL, "side_re must be > 0");
    if (p->npix_side < 1 || p->npix_side > 32768) return fail(MM_EINVAL, "npix_side must be in 1..32768");
    if (!finite(p->nrays_per_pix) || !(p->nrays_per_pix > 0.0)) return fail(MM_EINVAL, "nrays_per_pix must be > 0");
    if (!finite(p->smooth_frac) || p->smooth_frac < 0.0 || p->smooth_frac > 1.0) return fail(MM_EINVAL, "smooth_frac must be in [0, 1]");
    if (p->mass_model == MM_MASS_LOGNORMAL && (!finite(p->mass_mu) || !finite(p->mass_s) || p->mass_s < 0.0))
        return fail(MM_EINVAL, "lognormal mass parameters must be finite, s >= 0");
    const double margin = (p->shoot_margin > 0.0) ? p->shoot_margin : 1.5;
    if (!finite(margin)) return fail(MM_EINVAL, "shoot_margin must be finite");
    g->a = 1.0 - p->sigma - p->gamma;
    g->b = 1.0 - p->sigma + p->gamma;
    if (std::fabs(g->a) < 1e-3 || std::fabs(g->b) < 1e-3)
        return fail(MM_EINVAL, "ill-posed map: |1 - sigma -+ gamma| < 1e-3 (Eq. square diverges)");
    g->sigma_c = p->smooth_frac * p->sigma;
    g->sigma_star = (1.0 - p->smooth_frac) * p->sigma;
    g->pix = p->side_re / (double)p->npix_side;
    g->delta = g->pix / std::sqrt(p->nrays_per_pix);
    g->width = margin * p->side_re / std::fabs(g->a);
    g->height = margin * p->side_re / std::fabs(g->b);
    const double fx = std::ceil(g->width / g->delta), fy = std::ceil(g->height / g->delta);
    if (!(fx >= 1.0 && fy >= 1.0) || fx > 8388608.0 || fy > 8388608.0)
        return fail(MM_EINVAL, "ray grid must be 1..2^23 rays per side");
    if (g->width > 2e5 || g->height > 2e5) return fail(MM_EINVAL, "shot rectangle wider than 2e5 Einstein radii");
    g->nx = (long long)fx;
    g->ny = (long long)fy;
    g->mu_theory = 1.0 / ((1.0 - p->sigma) * (1.0 - p->sigma) - p->gamma * p->gamma);
    // lens field size (Eq. nstar with A = pi R^2) and disc radius (reading: half the
    // shot rectangle's diagonal plus 2 Einstein radii)
    g->mmean = (p->mass_model == MM_MASS_UNIT) ? 1.0 : std::exp(p->mass_mu + 0.5 * p->mass_s * p->mass_s);
    const double rule_r = 0.5 * margin * std::hypot(p->side_re / std::fabs(g->a), p->side_re / std::fabs(g->b)) + 2.0;
    if (p->nstar < 0 && !(p->disc_radius > 0.0)) {
        g->radius = rule_r;
        g->nstar = (g->sigma_star > 0.0) ? (long long)std::floor(g->sigma_star * g->radius * g->radius / g->mmean + 0.5) : 0;
    } else if (p->nstar >= 0 && !(p->disc_radius > 0.0)) {
        g->nstar = p->nstar;
        g->radius = (g->sigma_star > 0.0) ? std::sqrt((double)p->nstar * g->mmean / g->sigma_star) : rule_r;
    } else if (p->nstar < 0) {
        g->radius = p->disc_radius;
        g->nstar = (long long)std::floor(g->sigma_star * g->radius * g->radius / g->mmean + 0.5);
    } else {
        g->nstar = p->nstar;
        g->radius = p->disc_radius;
    }
    if (!finite(g->radius) || g->radius > 1e5) return fail(MM_EINVAL, "lens disc radius must be <= 1e5");
    if (g->nstar > 2000000000LL) return fail(MM_EINVAL, "nstar too large");
    // shot sub-rectangle
    const int64_t *r = p->ray_rect;
    if (r[0] == -1 && r[1] == -1 && r[2] == -1 && r[3] == -1) {
        g->i0 = 0; g->j0 = 0; g->ni = g->nx; g->nj = g->ny;
    } else {
        if (r[0] < 0 || r[1] < r[0] || r[1] > g->nx || r[2] < 0 || r[3] < r[2] || r[3] > g->ny)
            return fail(MM_EINVAL, "ray_rect outside the ray grid");
        g->i0 = r[0]; g->ni = r[1] - r[0]; g->j0 = r[2]; g->nj = r[3] - r[2];
    }
    if (p->ray_mode != MM_RAYS_LATTICE && p->ray_mode != MM_RAYS_RANDOM) return fail(MM_EINVAL, "bad ray_mode");
    if (p->ray_mode == MM_RAYS_RANDOM) {
        if (p->precision == MM_FAR32) return fail(MM_EINVAL, "random rays: MM_FP32C or MM_FP64 only");
        if (g->i0 % kTileX != 0 || g->j0 % kTileY != 0)
            return fail(MM_EINVAL, "random rays: ray_rect must start on the 64 x 32 tile grid");
    }
    g->tiles_x = (g->ni + kTileX - 1) / kTileX;
    g->tiles_y = (g->nj + kTileY - 1) / kTileY;
    return MM_OK;
}

// ------------------------------------------------------------------ arena ---

size_t DeviceArena::round(size_t bytes)
{
    if (bytes == 0) bytes = 1;
    const size_t q = bytes <= (1u << 20) ? 512 : (1u << 20);
    return (bytes + q - 1) / q * q;
}

bool DeviceArena::fits(size_t bytes) const
{
    // cached blocks can always be given back, so only live bytes count against room
    std::lock_guard<std::mutex> lk(mu_);
    return live_bytes_ + round(bytes) <= budget_;
}

int DeviceArena::alloc(size_t bytes, void **out)
{
    std::lock_guard<std::mutex> lk(mu_);
    const size_t r = round(bytes);
    auto it = cache_.lower_bound(r);
    if (it != cache_.end() && it->first <= 2 * r) {
        *out = it->second;
        live_[it->second] = it->first;
        live_bytes_ += it->first;
        cache_.erase(it);
        return MM_OK;
    }
    while (held_ + r > budget_ && !cache_.empty()) {
        auto big = std::prev(cache_.end());
        cudaFree(big->second);
        held_ -= big->first;
        cache_.erase(big);
    }
    if (held_ + r > budget_) return fail(MM_ENOMEM, "over the context's HBM budget");
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, r);
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (auto &kv : cache_) cudaFree(kv.second), held_ -= kv.first;
        cache_.clear();
        e = cudaMalloc(&p, r);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(MM_ENOMEM, "cudaMalloc failed");
        }
    }
    held_ += r;
    live_[p] = r;
    live_bytes_ += r;
    *out = p;
    return MM_OK;
}

void DeviceArena::free(void *p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu_);
    auto it = live_.find(p);
    if (it == live_.end()) return;
    cache_.emplace(it->second, p);
    live_bytes_ -= it->second;
    live_.erase(it);
}

void DeviceArena::release_all()
{
    std::lock_guard<std::mutex> lk(mu_);
    for (auto &kv : cache_) cudaFree(kv.second);
    for (auto &kv : live_) cudaFree(kv.first);
    cache_.clear();
    live_.clear();
    held_ = 0;
    live_bytes_ = 0;
}

LensSet::~LensSet()
{
    if (!arena) return;
    arena->free(dx); arena->free(dy); arena->free(dm); arena->free(lh); arena->free(lmf);
    tree.release(arena);
}

size_t LensSet::footprint(long long n)
{
    const long long pad = (n + kChunkLenses - 1) / kChunkLenses * kChunkLenses + kChunkLenses;
    return 3 * DeviceArena::round((size_t)std::max(n, 1LL) * 8) + DeviceArena::round((size_t)pad * 16) +
           DeviceArena::round((size_t)pad * 4);
}

MapObj::~MapObj()
{
    if (done) cudaEventDestroy(done);
    if (!arena) return;
    if (owns_outputs) {
        arena->free(counts);
        arena->free(totals);
    }
    arena->free(partial);
    arena->free(seg_done);
    far_release(*this);
}

void lens_split(const Geo &g, int precision, int *splits, long long *seg_lenses)
{
    *splits = 1;
    *seg_lenses = std::max(g.nstar, 1LL);
    const unsigned long long tiles = g.tiles();
    if (precision != MM_FP32C || tiles == 0 || tiles >= kSplitTargetItems || g.nstar <= 2 * kChunkLenses) return;
    const long long chunks = (g.nstar + kChunkLenses - 1) / kChunkLenses;
    const long long want = (long long)((kSplitTargetItems + tiles - 1) / tiles);
    const long long s = std::min(chunks, want);
    const long long seg_chunks = (chunks + s - 1) / s;
    *seg_lenses = seg_chunks * kChunkLenses;
    *splits = (int)((g.nstar + *seg_lenses - 1) / *seg_lenses);
    if (*splits <= 1) {
        *splits = 1;
        *seg_lenses = g.nstar;
    }
}

size_t MapObj::footprint(const mm_params *p, const Geo &g)
{
    int splits;
    long long seg;
    lens_split(g, p->precision, &splits, &seg);
    size_t b = DeviceArena::round((size_t)p->npix_side * (size_t)p->npix_side * 4) + DeviceArena::round(16);
    if (splits > 1)
        b += DeviceArena::round(g.tiles() * (size_t)splits * kTileRays * sizeof(float4)) +
             DeviceArena::round(g.tiles() * sizeof(unsigned));
    if (p->precision == MM_FAR32) {              // block series, near-list offsets and lists (estimated)
        const long long bt = far_block_for(g, *p, g.nstar, g.radius);
        const size_t blocks = (size_t)((g.ni + 64 * bt - 1) / (64 * bt)) * (size_t)((g.nj + 32 * bt - 1) / (32 * bt));
        const size_t stride = (size_t)((4 + 2 * (p->far_order - 1) + 3) & ~3);
        b += DeviceArena::round(blocks * stride * sizeof(float)) + DeviceArena::round((blocks + 1) * 8) +
             DeviceArena::round(blocks * 64 * sizeof(int)) + DeviceArena::round(sizeof(unsigned));
    }
    return b;
}

// ------------------------------------------------------------ lens sets ---

int upload_lenses(mm_ctx *ctx, const double *x, const double *y, const double *m, long long n, bool unit,
                  cudaStream_t s, std::shared_ptr<LensSet> *out)
{
    auto L = std::make_shared<LensSet>();
    L->arena = &ctx->arena;
    L->n = n;
    // padded to whole chunks, plus one extra chunk of null lenses
    L->n_pad = (n + kChunkLenses - 1) / kChunkLenses * kChunkLenses + kChunkLenses;
    L->unit_mass = unit;
    for (long long k = 0; k < n; ++k) L->radius = std::max(L->radius, std::hypot(x[k], y[k]));
    const size_t nb = (size_t)std::max(n, 1LL) * sizeof(double);
    int rc;
    if ((rc = ctx->arena.alloc(nb, (void **)&L->dx)) || (rc = ctx->arena.alloc(nb, (void **)&L->dy)) ||
        (rc = ctx->arena.alloc(nb, (void **)&L->dm)) ||
        (rc = ctx->arena.alloc((size_t)L->n_pad * sizeof(float4), (void **)&L->lh)) ||
        (rc = ctx->arena.alloc((size_t)L->n_pad * sizeof(float), (void **)&L->lmf)))
        return rc;
    if (n > 0) {
        MM_CUDA(cudaMemcpyAsync(L->dx, x, (size_t)n * 8, cudaMemcpyHostToDevice, s));
        MM_CUDA(cudaMemcpyAsync(L->dy, y, (size_t)n * 8, cudaMemcpyHostToDevice, s));
        MM_CUDA(cudaMemcpyAsync(L->dm, m, (size_t)n * 8, cudaMemcpyHostToDevice, s));
    }
    MM_CUDA(launch_prepare_lenses(L->dx, L->dy, L->dm, n, L->n_pad, L->lh, L->lmf, s));
    *out = L;
    return MM_OK;
}

int make_lenses_from_params(mm_ctx *ctx, const mm_params *p, const Geo &g, cudaStream_t s,
                            std::shared_ptr<LensSet> *out)
{
    std::vector<double> x, y, m;
    generate_field(p->seed, g.nstar, g.radius, p->mass_model, p->mass_mu, p->mass_s, x, y, m);
    int rc = upload_lenses(ctx, x.data(), y.data(), m.data(), g.nstar, p->mass_model == MM_MASS_UNIT, s, out);
    if (rc) return rc;
    (*out)->radius = g.radius;           // the disc the field fills (as mm_geometry_of reports it)
    MM_CUDA(cudaStreamSynchronize(s));   // host vectors go out of scope
    return MM_OK;
}

static uint64_t new_handle(mm_ctx *ctx) { return ctx->next_handle.fetch_add(1); }

// ------------------------------------------------------------------ maps ---

static size_t map_bytes(const mm_params *p) { return (size_t)p->npix_side * (size_t)p->npix_side * 4; }

int alloc_map(mm_ctx *ctx, const mm_params *p, const Geo &g, std::shared_ptr<LensSet> lenses, cudaStream_t s,
              std::shared_ptr<MapObj> *out, const MapObj *into)
{
    auto M = std::make_shared<MapObj>();
    M->arena = &ctx->arena;
    M->p = *p;
    M->g = g;
    M->lenses = std::move(lenses);
    M->owns_outputs = !into;
    int rc;
    if (into) {
        // a part of another map: its counts, totals and variant, and the lens split of the
        // whole ray grid, so that the part's tiles sum their lenses as a one-shot map's do
        M->counts = into->counts;
        M->totals = into->totals;
        Geo whole = g;
        whole.nstar = M->lenses->n;
        whole.tiles_x = (g.nx + kTileX - 1) / kTileX;
        whole.tiles_y = (g.ny + kTileY - 1) / kTileY;
        lens_split(whole, p->precision, &M->splits, &M->seg_lenses);
    } else {
        if ((rc = ctx->arena.alloc(map_bytes(p), (void **)&M->counts)) ||
            (rc = ctx->arena.alloc(2 * sizeof(unsigned long long), (void **)&M->totals)))
            return rc;
        Geo gl = g;
        gl.nstar = M->lenses->n;
        lens_split(gl, p->precision, &M->splits, &M->seg_lenses);
    }
    if (M->splits > 1) {
        if ((rc = ctx->arena.alloc(g.tiles() * (size_t)M->splits * kTileRays * sizeof(float4), (void **)&M->partial)) ||
            (rc = ctx->arena.alloc(g.tiles() * sizeof(unsigned), (void **)&M->seg_done)))
            return rc;
        MM_CUDA(cudaMemsetAsync(M->seg_done, 0, g.tiles() * sizeof(unsigned), s));
    }
    MM_CUDA(cudaEventCreateWithFlags(&M->done, cudaEventDisableTiming));
    if (!into) {
        MM_CUDA(cudaMemsetAsync(M->counts, 0, map_bytes(p), s));
        MM_CUDA(cudaMemsetAsync(M->totals, 0, 2 * sizeof(unsigned long long), s));
    }
    M->variant = into ? into->variant : choose_variant(ctx, M->lenses->unit_mass, M->lenses->n);
    M->shot_total = (unsigned long long)g.ni * (unsigned long long)g.nj;
    *out = M;
    return MM_OK;
}

static void split_ff(double v, float *h, float *l)
{
    *h = (float)v;
    *l = (float)(v - (double)*h);
}

void fill_desc(const MapObj &m, MapDesc *d)
{
    const Geo &g = m.g;
    std::memset(d, 0, sizeof(*d));
    d->delta = g.delta;
    d->half_nx = 0.5 * (double)g.nx;
    d->half_ny = 0.5 * (double)g.ny;
    d->nx = g.nx;
    d->ny = g.ny;
    d->i0 = g.i0; d->j0 = g.j0; d->ni = g.ni; d->nj = g.nj;
    d->tiles_x = g.tiles_x;
    d->one_m_gamma = 1.0 - m.p.gamma;
    d->one_p_gamma = 1.0 + m.p.gamma;
    d->sigma_c = g.sigma_c;
    d->half_side = 0.5 * m.p.side_re;
    d->pix = g.pix;
    const double a1 = (1.0 - m.p.gamma) - g.sigma_c, a2 = (1.0 + m.p.gamma) - g.sigma_c;
    split_ff(a1 * g.delta / (2.0 * g.pix), &d->ax_h, &d->ax_l);
    split_ff(a2 * g.delta / (2.0 * g.pix), &d->ay_h, &d->ay_l);
    split_ff((double)m.p.npix_side / m.p.side_re, &d->ip_h, &d->ip_l);
    d->half_n = 0.5f * (float)m.p.npix_side;
    split_ff(g.delta, &d->delta_f, &d->delta_l);
    d->nside = m.p.npix_side;
    d->unit_mass = m.lenses->unit_mass ? 1 : 0;
    d->variant = m.variant;
    d->precision = m.p.precision;
    d->nstar = m.lenses->n;
    d->lx = m.lenses->dx; d->ly = m.lenses->dy; d->lm = m.lenses->dm;
    d->lh = m.lenses->lh; d->lmf = m.lenses->lmf;
    d->counts = m.counts;
    d->totals = m.totals;
    d->lens_splits = m.splits;
    d->seg_lenses = m.splits > 1 ? m.seg_lenses : std::max(m.lenses->n, 1LL);
    d->partial = m.partial;
    d->seg_done = m.seg_done;
    d->random_rays = m.p.ray_mode == MM_RAYS_RANDOM ? 1 : 0;
    d->ray_seed = m.p.ray_seed;
}

static int class_key(bool unit_mass, long long nstar)
{
    int b = 0;
    while (b < 40 && (1LL << b) <= nstar) ++b;
    return (unit_mass ? 0 : 1000) + b;
}

int choose_variant(mm_ctx *ctx, bool unit_mass, long long nstar)
{
    if (ctx->forced_variant >= 0) return ctx->forced_variant;
    auto it = ctx->tuned.find(class_key(unit_mass, nstar));
    if (it != ctx->tuned.end()) return it->second;
    return default_variant(unit_mass);
}

uint64_t register_map(mm_ctx *ctx, std::shared_ptr<MapObj> m)
{
    const uint64_t h = new_handle(ctx);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->maps[h] = std::move(m);
    return h;
}

int scratch_reserve(mm_ctx *ctx, LaunchScratch *sc, int n_maps)
{
    if (!sc->d_hdr) {
        MM_CUDA(cudaMalloc(&sc->d_hdr, sizeof(WorkHeader)));
        MM_CUDA(cudaMalloc(&sc->d_counter, sizeof(unsigned long long)));
        MM_CUDA(cudaMalloc(&sc->d_check, sizeof(unsigned int)));
        MM_CUDA(cudaMemset(sc->d_check, 0, sizeof(unsigned int)));
        MM_CUDA(cudaMallocHost(&sc->h_hdr, sizeof(WorkHeader)));
    }
    if (n_maps > sc->cap) {
        const int cap = std::max(n_maps, std::max(64, 2 * sc->cap));
        if (sc->d_maps) cudaFree(sc->d_maps);
        if (sc->h_maps) cudaFreeHost(sc->h_maps);
        if (sc->d_far) cudaFree(sc->d_far);
        if (sc->h_far) cudaFreeHost(sc->h_far);
        sc->d_maps = nullptr;
        sc->h_maps = nullptr;
        sc->d_far = nullptr;
        sc->h_far = nullptr;
        sc->cap = 0;
        MM_CUDA(cudaMalloc(&sc->d_maps, (size_t)cap * sizeof(MapDesc)));
        MM_CUDA(cudaMallocHost(&sc->h_maps, (size_t)cap * sizeof(MapDesc)));
        MM_CUDA(cudaMalloc(&sc->d_far, (size_t)cap * sizeof(FarDesc)));
        MM_CUDA(cudaMallocHost(&sc->h_far, (size_t)cap * sizeof(FarDesc)));
        sc->cap = cap;
    }
    (void)ctx;
    return MM_OK;
}

void scratch_free(mm_ctx *ctx, LaunchScratch *sc)
{
    (void)ctx;
    if (sc->d_hdr) cudaFree(sc->d_hdr);
    if (sc->d_maps) cudaFree(sc->d_maps);
    if (sc->d_counter) cudaFree(sc->d_counter);
    if (sc->d_check) cudaFree(sc->d_check);
    if (sc->h_hdr) cudaFreeHost(sc->h_hdr);
    if (sc->h_maps) cudaFreeHost(sc->h_maps);
    if (sc->d_far) cudaFree(sc->d_far);
    if (sc->h_far) cudaFreeHost(sc->h_far);
    *sc = LaunchScratch{};
}

// Launch one precision group of maps as one persistent launch on stream s,
// bracketed by ctx->ev0/ev1. Maps are ordered by decreasing per-tile cost. For
// MM_FAR32 the bracket also holds each map's block preparation.
static int launch_group(mm_ctx *ctx, std::vector<MapObj *> &group, int precision, const DumpArgs *dump,
                        unsigned long long dump_items, cudaStream_t s, float *ms)
{
    const bool fp64 = precision == MM_FP64, far = precision == MM_FAR32;
    if (group.empty()) return MM_OK;
    LaunchScratch *sc = &ctx->scratch;
    int rc = scratch_reserve(ctx, sc, (int)group.size());
    if (rc) return rc;
    std::stable_sort(group.begin(), group.end(), [](const MapObj *a, const MapObj *b) {
        const long long ca = a->splits > 1 ? a->seg_lenses : a->lenses->n;
        const long long cb = b->splits > 1 ? b->seg_lenses : b->lenses->n;
        return ca > cb;                                  // most expensive work items first
    });
    unsigned long long total = 0;
    for (size_t k = 0; k < group.size(); ++k) {
        MapDesc *d = &sc->h_maps[k];
        fill_desc(*group[k], d);
        d->item_begin = total;
        d->item_first = 0;
        d->item_count = group[k]->items();
        total += d->item_count;
    }
    // a debug dump covers dump_items tiles of one map, each with all its lens segments
    sc->h_hdr->total_work = dump ? dump_items * (unsigned long long)group[0]->splits : total;
    sc->h_hdr->n_maps = (int)group.size();
    MM_CUDA(cudaMemcpyAsync(sc->d_hdr, sc->h_hdr, sizeof(WorkHeader), cudaMemcpyHostToDevice, s));
    MM_CUDA(cudaMemcpyAsync(sc->d_maps, sc->h_maps, group.size() * sizeof(MapDesc), cudaMemcpyHostToDevice, s));
    MM_CUDA(cudaMemsetAsync(sc->d_counter, 0, sizeof(unsigned long long), s));
    LaunchArgs a{};
    a.hdr = sc->d_hdr;
    a.maps = sc->d_maps;
    a.work_counter = sc->d_counter;
    a.check = sc->d_check;
    if (dump) a.dump = *dump;
#ifdef MM_CHECKS
    MM_CUDA(cudaMemsetAsync(sc->d_check, 0, sizeof(unsigned int), s));
#endif
    const unsigned long long work = sc->h_hdr->total_work;
    // a launch holds maps of one ray mode (the batch groups them; the other callers launch one map)
    const bool random = group[0]->p.ray_mode == MM_RAYS_RANDOM;
    for (const MapObj *m : group)
        if ((m->p.ray_mode == MM_RAYS_RANDOM) != random) return fail(MM_EINVAL, "a launch mixes ray modes");
    const long long cap = (long long)ctx->sms * (far      ? far_ctas_per_sm()
                                                 : random ? shoot_ctas_per_sm(fp64, kRandomLayout)
                                                          : shoot_ctas_per_sm(fp64, ctx->layout));
    const int grid = (int)std::max(1LL, std::min((long long)work, cap));
    MM_CUDA(cudaEventRecord(ctx->ev0, s));
    unsigned long long far_items = 0;
    if (far) {
        for (size_t k = 0; k < group.size(); ++k) {
            if ((rc = far_prepare(ctx, *group[k], s, sc->d_check))) return rc;
            group[k]->far.item_begin = far_items;
            far_items += group[k]->far.items;
            sc->h_far[k] = group[k]->far;
            ctx->last_launches += group[k]->far.nblocks > 0 ? 3 : 0;
        }
        MM_CUDA(cudaMemcpyAsync(sc->d_far, sc->h_far, group.size() * sizeof(FarDesc), cudaMemcpyHostToDevice, s));
    }
    bool split = false;
    for (const MapObj *m : group) split = split || m->splits > 1;
    if (work > 0) {
        if (far && !dump)
            MM_CUDA(launch_shoot_far(a, sc->d_far, far_items, (int)std::max(1LL, std::min((long long)far_items, cap)),
                                     false, s));
        else if (far) MM_CUDA(launch_shoot_far(a, sc->d_far, 0, grid, true, s));
        else if (fp64) MM_CUDA(launch_shoot_fp64(a, grid, dump != nullptr, s));
        else if (random) MM_CUDA(launch_shoot_fp32_random(a, grid, dump != nullptr, split, s));
        else MM_CUDA(launch_shoot_fp32(a, ctx->layout, grid, dump != nullptr, split, s));
    }
    MM_CUDA(cudaEventRecord(ctx->ev1, s));
    MM_CUDA(cudaEventSynchronize(ctx->ev1));     // pinned scratch is reused by the next call
    float t = 0.f;
    MM_CUDA(cudaEventElapsedTime(&t, ctx->ev0, ctx->ev1));
    *ms = t;
    ctx->last_ms = t;
    ctx->last_launches += work > 0 ? 1 : 0;
#ifdef MM_CHECKS
    unsigned bad = 0;
    MM_CUDA(cudaMemcpy(&bad, sc->d_check, sizeof(bad), cudaMemcpyDeviceToHost));
    if (bad) return fail(MM_EDEVICE, "bounds check failed at site " + std::to_string(bad));
#endif
    if (far) {
        for (MapObj *m : group) {                 // the largest tail bound of the map's blocks
            unsigned bits = 0;
            MM_CUDA(cudaMemcpy(&bits, m->far_bmax, sizeof(bits), cudaMemcpyDeviceToHost));
            float b;
            std::memcpy(&b, &bits, sizeof(b));
            m->far_bound = std::max(m->far_bound, (double)b);
        }
    }
    return MM_OK;
}

static std::shared_ptr<LensSet> find_lenses(mm_ctx *ctx, mm_lenses h)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->lenses.find(h);
    return it == ctx->lenses.end() ? nullptr : it->second;
}

static std::shared_ptr<MapObj> find_map(mm_ctx *ctx, mm_map h)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->maps.find(h);
    return it == ctx->maps.end() ? nullptr : it->second;
}

// Shared preparation of one map of a synchronous call.
static int prepare_map(mm_ctx *ctx, mm_lenses lh, const mm_params *p, std::shared_ptr<MapObj> *out)
{
    Geo g;
    int rc = compute_geo(p, &g);
    if (rc) return rc;
    std::shared_ptr<LensSet> L;
    if (lh) {
        L = find_lenses(ctx, lh);
        if (!L) return fail(MM_ENOTFOUND, "unknown lens set");
        g.nstar = L->n;
    } else {
        rc = make_lenses_from_params(ctx, p, g, ctx->stream, &L);
        if (rc) return rc;
    }
    return alloc_map(ctx, p, g, L, ctx->stream, out);
}

}  // namespace mm

using namespace mm;

// ================================================================ C ABI ====

// FP64 per-ray deflections: every FP64 ray is computed independently of its tile, so the
// listed rays run one thread each (the map kernel's per-ray arithmetic) instead of
// through their whole tiles.
static int debug_rays_fp64(mm_ctx *ctx, const MapObj &M, const int64_t *ray_i, const int64_t *ray_j, int64_t n,
                           double *alpha_out, int64_t *pixel_out)
{
    struct Tmp {
        DeviceArena *a;
        std::vector<void *> v;
        ~Tmp() { for (void *p : v) a->free(p); }
    } tmp{&ctx->arena, {}};
    auto dalloc = [&](size_t bytes, void **out) -> int {
        int r = ctx->arena.alloc(bytes, out);
        if (!r) tmp.v.push_back(*out);
        return r;
    };
    long long *d_i, *d_j, *d_pixel;
    double *d_alpha;
    int rc;
    if ((rc = dalloc((size_t)n * 8, (void **)&d_i)) || (rc = dalloc((size_t)n * 8, (void **)&d_j)) ||
        (rc = dalloc((size_t)n * 16, (void **)&d_alpha)) || (rc = dalloc((size_t)n * 8, (void **)&d_pixel)))
        return rc;
    MapDesc d;
    fill_desc(M, &d);
    cudaStream_t s = ctx->stream;
    static_assert(sizeof(long long) == sizeof(int64_t), "ray indices are 64-bit");
    MM_CUDA(cudaMemcpyAsync(d_i, ray_i, (size_t)n * 8, cudaMemcpyHostToDevice, s));
    MM_CUDA(cudaMemcpyAsync(d_j, ray_j, (size_t)n * 8, cudaMemcpyHostToDevice, s));
    cudaEvent_t e0 = ctx->ev0, e1 = ctx->ev1;
    MM_CUDA(cudaEventRecord(e0, s));
    MM_CUDA(launch_rays_fp64(d, d_i, d_j, n, d_alpha, d_pixel, s));
    MM_CUDA(cudaEventRecord(e1, s));
    if (alpha_out) MM_CUDA(cudaMemcpyAsync(alpha_out, d_alpha, (size_t)n * 16, cudaMemcpyDeviceToHost, s));
    if (pixel_out) MM_CUDA(cudaMemcpyAsync(pixel_out, d_pixel, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    MM_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    MM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    ctx->last_ms = ms;
    ctx->last_launches = 1;
    return MM_OK;
}

extern "C" {

const char *mm_strerror(int code)
{
    switch (code) {
    case MM_OK: return "ok";
    case MM_EINVAL: return "invalid argument";
    case MM_ENOMEM: return "out of device memory budget";
    case MM_EBUSY: return "busy";
    case MM_ENOTFOUND: return "handle not found";
    case MM_ETIMEDOUT: return "timed out";
    case MM_EDEVICE: return "CUDA device error";
    case MM_EAGAIN: return "not finished";
    case MM_ECANCELED: return "cancelled";
    default: return "unknown error";
    }
}

const char *mm_last_error(void) { return g_last_error.c_str(); }

int mm_init(mm_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream)
{
    if (!out) return fail(MM_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
        cudaGetLastError();
        return fail(MM_EDEVICE, "no CUDA device");
    }
    if (device < 0 || device >= ndev) return fail(MM_EINVAL, "bad device index");
    MM_CUDA(cudaSetDevice(device));
    cudaDeviceProp prop;
    MM_CUDA(cudaGetDeviceProperties(&prop, device));
    auto *ctx = new mm_ctx();
    ctx->device = device;
    ctx->sms = prop.multiProcessorCount;
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete ctx; return cuda_fail(e, "cudaStreamCreate"); }
        ctx->own_stream = true;
    }
    size_t freeb = 0, totalb = 0;
    cudaMemGetInfo(&freeb, &totalb);
    ctx->arena.init(hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)freeb));
    if (cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return fail(MM_EDEVICE, "cudaEventCreate failed");
    }
    *out = ctx;
    return MM_OK;
}

int mm_destroy(mm_ctx *ctx)
{
    if (!ctx) return MM_OK;
    cudaSetDevice(ctx->device);
    server_stop(ctx);
    cudaStreamSynchronize(ctx->stream);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->maps.clear();
        ctx->lenses.clear();
    }
    scratch_free(ctx, &ctx->scratch);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    ctx->arena.release_all();
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return MM_OK;
}

int mm_params_default(mm_params *p)
{
    if (!p) return fail(MM_EINVAL, "params is NULL");
    std::memset(p, 0, sizeof(*p));
    p->shoot_margin = 1.5;
    p->precision = MM_FP32C;
    p->nstar = -1;
    p->disc_radius = 0.0;
    p->mass_model = MM_MASS_UNIT;
    p->mass_mu = 0.0;
    p->mass_s = 0.5;
    p->seed = 1;
    for (int k = 0; k < 4; ++k) p->ray_rect[k] = -1;
    p->far_order = 10;
    p->far_ratio = 0.15;
    p->far_block = 0;
    p->far_group_order = -1;
    p->far_group_theta = 0.3;
    p->far_group_leaf = 64;
    p->ray_mode = MM_RAYS_LATTICE;
    p->ray_seed = 1;
    return MM_OK;
}

int mm_geometry_of(const mm_params *p, mm_geometry *out)
{
    if (!out) return fail(MM_EINVAL, "out is NULL");
    Geo g;
    int rc = compute_geo(p, &g);
    if (rc) return rc;
    out->pix = g.pix;
    out->delta = g.delta;
    out->width = g.width;
    out->height = g.height;
    out->nx = g.nx;
    out->ny = g.ny;
    out->nstar = g.nstar;
    out->disc_radius = g.radius;
    out->mu_theory = g.mu_theory;
    out->far_block = far_block_for(g, *p, g.nstar, g.radius);
    out->far_group = p->precision == MM_FAR32 ? far_group_for(g, *p, g.nstar, g.radius) : 0;
    return MM_OK;
}

int mm_create_lenses(mm_ctx *ctx, const mm_params *p, mm_lenses *out)
{
    NvtxRange nvtx_("mm_create_lenses");
    if (!ctx || !out) return fail(MM_EINVAL, "null argument");
    Geo g;
    int rc = compute_geo(p, &g);
    if (rc) return rc;
    cudaSetDevice(ctx->device);
    std::shared_ptr<LensSet> L;
    rc = make_lenses_from_params(ctx, p, g, ctx->stream, &L);
    if (rc) return rc;
    const uint64_t h = new_handle(ctx);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->lenses[h] = L;
    *out = h;
    return MM_OK;
}

int mm_create_lenses_from(mm_ctx *ctx, const double *x, const double *y, const double *m, int64_t n, mm_lenses *out)
{
    NvtxRange nvtx_("mm_create_lenses_from");
    if (!ctx || !out || n < 0 || (n > 0 && (!x || !y || !m))) return fail(MM_EINVAL, "bad lens arrays");
    bool unit = true;
    for (int64_t k = 0; k < n; ++k) {
        if (!std::isfinite(x[k]) || !std::isfinite(y[k]) || !std::isfinite(m[k]) || m[k] < 0.0)
            return fail(MM_EINVAL, "lens coordinates must be finite and masses >= 0");
        if (std::fabs(x[k]) > 1e5 || std::fabs(y[k]) > 1e5) return fail(MM_EINVAL, "lens coordinate beyond 1e5");
        if (m[k] != 1.0) unit = false;
    }
    cudaSetDevice(ctx->device);
    std::shared_ptr<LensSet> L;
    int rc = upload_lenses(ctx, x, y, m, n, unit, ctx->stream, &L);
    if (rc) return rc;
    MM_CUDA(cudaStreamSynchronize(ctx->stream));
    const uint64_t h = new_handle(ctx);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->lenses[h] = L;
    *out = h;
    return MM_OK;
}

int mm_lenses_count(mm_ctx *ctx, mm_lenses h, int64_t *n)
{
    if (!ctx || !n) return fail(MM_EINVAL, "null argument");
    auto L = find_lenses(ctx, h);
    if (!L) return fail(MM_ENOTFOUND, "unknown lens set");
    *n = L->n;
    return MM_OK;
}

int mm_lenses_fetch(mm_ctx *ctx, mm_lenses h, double *x, double *y, double *m, int64_t n)
{
    if (!ctx) return fail(MM_EINVAL, "null context");
    auto L = find_lenses(ctx, h);
    if (!L) return fail(MM_ENOTFOUND, "unknown lens set");
    if (n != L->n) return fail(MM_EINVAL, "n does not match the lens set");
    cudaSetDevice(ctx->device);
    if (n > 0) {
        if (x) MM_CUDA(cudaMemcpyAsync(x, L->dx, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream));
        if (y) MM_CUDA(cudaMemcpyAsync(y, L->dy, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream));
        if (m) MM_CUDA(cudaMemcpyAsync(m, L->dm, (size_t)n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    }
    MM_CUDA(cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}

int mm_release_lenses(mm_ctx *ctx, mm_lenses h)
{
    if (!ctx) return fail(MM_EINVAL, "null context");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->lenses.erase(h) == 0) return fail(MM_ENOTFOUND, "unknown lens set");
    return MM_OK;
}

int mm_shoot(mm_ctx *ctx, mm_lenses lenses, const mm_params *p, mm_map *out)
{
    NvtxRange nvtx_("mm_shoot");
    if (!ctx || !out) return fail(MM_EINVAL, "null argument");
    cudaSetDevice(ctx->device);
    std::shared_ptr<MapObj> M;
    int rc = prepare_map(ctx, lenses, p, &M);
    if (rc) return rc;
    ctx->last_launches = 0;
    std::vector<MapObj *> group{M.get()};
    float ms = 0.f;
    rc = launch_group(ctx, group, p->precision, nullptr, 0, ctx->stream, &ms);
    if (rc) return rc;
    MM_CUDA(cudaEventRecord(M->done, ctx->stream));
    M->seconds = ms * 1e-3;
    *out = register_map(ctx, M);
    return MM_OK;
}

int mm_shoot_batch(mm_ctx *ctx, int32_t n, const mm_lenses *lenses, const mm_params *params, mm_map *maps_out)
{
    NvtxRange nvtx_("mm_shoot_batch");
    if (!ctx || n < 0 || (n > 0 && (!params || !maps_out))) return fail(MM_EINVAL, "bad batch arguments");
    cudaSetDevice(ctx->device);
    std::vector<std::shared_ptr<MapObj>> objs((size_t)n);
    for (int k = 0; k < n; ++k) {
        int rc = prepare_map(ctx, lenses ? lenses[k] : 0, &params[k], &objs[(size_t)k]);
        if (rc) return rc;
    }
    ctx->last_launches = 0;
    // one launch per precision (MM_FP32C, MM_FP64, MM_FAR32) and ray mode (lattice, random)
    auto group_of = [](const MapObj &o) { return o.p.precision + (o.p.ray_mode == MM_RAYS_RANDOM ? 3 : 0); };
    std::vector<MapObj *> groups[6];
    for (auto &o : objs) groups[group_of(*o)].push_back(o.get());
    float ms[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    ctx->last_ms = 0.0;
    for (int k = 0; k < 6; ++k) {
        int rc = launch_group(ctx, groups[k], k % 3, nullptr, 0, ctx->stream, &ms[k]);
        if (rc) return rc;
    }
    ctx->last_ms = ms[0] + ms[1] + ms[2] + ms[3] + ms[4] + ms[5];
    for (int k = 0; k < n; ++k) {
        auto &o = objs[(size_t)k];
        o->seconds = ms[group_of(*o)] * 1e-3;
        MM_CUDA(cudaEventRecord(o->done, ctx->stream));
        maps_out[k] = register_map(ctx, o);
    }
    return MM_OK;
}

int mm_shoot_into(mm_ctx *ctx, mm_lenses lenses, const mm_params *p, mm_map map)
{
    NvtxRange nvtx_("mm_shoot_into");
    if (!ctx || !p) return fail(MM_EINVAL, "null argument");
    auto T = find_map(ctx, map);
    if (!T) return fail(MM_ENOTFOUND, "unknown map");
    const mm_params &q = T->p;
    const double margin_p = p->shoot_margin > 0 ? p->shoot_margin : 1.5, margin_q = q.shoot_margin > 0 ? q.shoot_margin : 1.5;
    if (p->sigma != q.sigma || p->gamma != q.gamma || p->smooth_frac != q.smooth_frac || p->side_re != q.side_re ||
        p->npix_side != q.npix_side || p->nrays_per_pix != q.nrays_per_pix || margin_p != margin_q ||
        p->precision != q.precision || p->ray_mode != q.ray_mode ||
        (p->ray_mode == MM_RAYS_RANDOM && p->ray_seed != q.ray_seed) ||
        (p->precision == MM_FAR32 &&
         (p->far_order != q.far_order || p->far_ratio != q.far_ratio || p->far_block != q.far_block ||
          p->far_group_order != q.far_group_order || p->far_group_theta != q.far_group_theta ||
          p->far_group_leaf != q.far_group_leaf)))
        return fail(MM_EINVAL, "parameters differ from the map's (only ray_rect may change)");
    cudaSetDevice(ctx->device);
    std::shared_ptr<LensSet> L = T->lenses;
    if (lenses) {
        L = find_lenses(ctx, lenses);
        if (!L) return fail(MM_ENOTFOUND, "unknown lens set");
        if (L->n != T->lenses->n) return fail(MM_EINVAL, "lens set differs in size from the map's");
    }
    Geo g;
    int rc = compute_geo(p, &g);
    if (rc) return rc;
    g.nstar = L->n;
    std::shared_ptr<MapObj> M;
    if ((rc = alloc_map(ctx, p, g, L, ctx->stream, &M, T.get()))) return rc;
    MM_CUDA(cudaStreamWaitEvent(ctx->stream, T->done, 0));
    ctx->last_launches = 0;
    std::vector<MapObj *> group{M.get()};
    float ms = 0.f;
    rc = launch_group(ctx, group, p->precision, nullptr, 0, ctx->stream, &ms);
    if (rc) return rc;
    MM_CUDA(cudaEventRecord(T->done, ctx->stream));
    T->shot_total += M->shot_total;
    T->seconds += ms * 1e-3;
    T->far_bound = std::max(T->far_bound, M->far_bound);
    return MM_OK;
}

int mm_map_restore(mm_ctx *ctx, mm_lenses lenses, const mm_params *p, const uint32_t *host_counts, size_t n_elems,
                   const mm_stats *st, mm_map *out)
{
    NvtxRange nvtx_("mm_map_restore");
    if (!ctx || !p || !host_counts || !st || !out) return fail(MM_EINVAL, "null argument");
    mm_params q = *p;
    for (int k = 0; k < 4; ++k) q.ray_rect[k] = 0;      // a map of no rays, then the checkpoint's counts
    const size_t npix = (size_t)q.npix_side * (size_t)q.npix_side;
    if (q.npix_side > 0 && n_elems != npix) return fail(MM_EINVAL, "n_elems must equal N_side^2");
    cudaSetDevice(ctx->device);
    std::shared_ptr<MapObj> M;
    int rc = prepare_map(ctx, lenses, &q, &M);
    if (rc) return rc;
    if (st->nstar != M->lenses->n || st->nx != (uint64_t)M->g.nx || st->ny != (uint64_t)M->g.ny)
        return fail(MM_EINVAL, "checkpoint was taken with other parameters or another lens count");
    unsigned long long sum = 0;
    for (size_t k = 0; k < npix; ++k) sum += host_counts[k];
    if (sum != st->rays_in || st->rays_in + st->rays_out != st->rays_shot ||
        st->rays_shot > (uint64_t)M->g.nx * (uint64_t)M->g.ny)
        return fail(MM_EINVAL, "checkpoint counts and totals disagree");
    const unsigned long long tot[2] = {st->rays_in, st->rays_out};
    MM_CUDA(cudaMemcpyAsync(M->counts, host_counts, npix * 4, cudaMemcpyHostToDevice, ctx->stream));
    MM_CUDA(cudaMemcpyAsync(M->totals, tot, sizeof(tot), cudaMemcpyHostToDevice, ctx->stream));
    MM_CUDA(cudaEventRecord(M->done, ctx->stream));
    MM_CUDA(cudaStreamSynchronize(ctx->stream));        // host buffers may go as soon as this returns
    M->shot_total = st->rays_shot;
    M->seconds = st->seconds;
    M->far_bound = st->far_bound;
    *out = register_map(ctx, M);
    return MM_OK;
}

int mm_map_fetch(mm_ctx *ctx, mm_map map, uint32_t *host_counts, size_t n_elems, mm_stats *st)
{
    NvtxRange nvtx_("mm_map_fetch");
    if (!ctx) return fail(MM_EINVAL, "null context");
    auto M = find_map(ctx, map);
    if (!M) return fail(MM_ENOTFOUND, "unknown map");
    const size_t npix = (size_t)M->p.npix_side * (size_t)M->p.npix_side;
    if (host_counts && n_elems != npix) return fail(MM_EINVAL, "n_elems must equal N_side^2");
    cudaSetDevice(ctx->device);
    MM_CUDA(cudaStreamWaitEvent(ctx->stream, M->done, 0));
    unsigned long long tot[2] = {0, 0};
    if (host_counts) MM_CUDA(cudaMemcpyAsync(host_counts, M->counts, npix * 4, cudaMemcpyDeviceToHost, ctx->stream));
    MM_CUDA(cudaMemcpyAsync(tot, M->totals, sizeof(tot), cudaMemcpyDeviceToHost, ctx->stream));
    MM_CUDA(cudaStreamSynchronize(ctx->stream));
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->rays_shot = M->shot_total;
        st->rays_in = tot[0];
        st->rays_out = tot[1];
        st->interactions = st->rays_shot * (uint64_t)M->lenses->n;
        st->nx = (uint64_t)M->g.nx;
        st->ny = (uint64_t)M->g.ny;
        st->nstar = M->lenses->n;
        st->seconds = M->seconds;
        st->mu_mean = (double)tot[0] / ((double)npix * M->p.nrays_per_pix);
        st->lens_splits = M->splits;
        st->far_bound = M->far_bound;
        st->far_block = M->p.precision == MM_FAR32 ? far_block_for(M->g, M->p, M->lenses->n, M->lenses->radius) : 0;
        st->far_group = M->p.precision == MM_FAR32 ? far_group_for(M->g, M->p, M->lenses->n, M->lenses->radius) : 0;
    }
    return MM_OK;
}

int mm_map_device_ptr(mm_ctx *ctx, mm_map map, void **dptr, size_t *n_elems)
{
    if (!ctx || !dptr) return fail(MM_EINVAL, "null argument");
    auto M = find_map(ctx, map);
    if (!M) return fail(MM_ENOTFOUND, "unknown map");
    *dptr = M->counts;
    if (n_elems) *n_elems = (size_t)M->p.npix_side * (size_t)M->p.npix_side;
    return MM_OK;
}

int mm_release_map(mm_ctx *ctx, mm_map map)
{
    if (!ctx) return fail(MM_EINVAL, "null context");
    std::shared_ptr<MapObj> M;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->maps.find(map);
        if (it == ctx->maps.end()) return fail(MM_ENOTFOUND, "unknown map");
        M = it->second;
        ctx->maps.erase(it);
    }
    cudaSetDevice(ctx->device);
    cudaEventSynchronize(M->done);   // device may still write it; free only when done
    return MM_OK;
}

int mm_debug_deflect(mm_ctx *ctx, mm_lenses lenses, const mm_params *p, const int64_t *ray_i, const int64_t *ray_j,
                     int64_t n, double *alpha_out, int64_t *pixel_out)
{
    NvtxRange nvtx_("mm_debug_deflect");
    if (!ctx || n < 0 || (n > 0 && (!ray_i || !ray_j))) return fail(MM_EINVAL, "bad ray arrays");
    if (n > (1LL << 28)) return fail(MM_EINVAL, "too many rays for one debug call");
    cudaSetDevice(ctx->device);
    std::shared_ptr<MapObj> M;
    int rc = prepare_map(ctx, lenses, p, &M);
    if (rc) return rc;
    if (n == 0) return MM_OK;
    const Geo &g = M->g;
    for (int64_t k = 0; k < n; ++k)
        if (ray_i[k] < g.i0 || ray_j[k] < g.j0 || ray_i[k] >= g.i0 + g.ni || ray_j[k] >= g.j0 + g.nj)
            return fail(MM_EINVAL, "ray outside the shot grid");
    if (p->precision == MM_FP64) return debug_rays_fp64(ctx, *M, ray_i, ray_j, n, alpha_out, pixel_out);
    // group the requested rays by the tile the map kernel would put them in,
    // sorted by (tile, local ray index) so the kernel can binary-search
    std::vector<std::pair<unsigned long long, int>> key((size_t)n);
    for (int64_t k = 0; k < n; ++k) {
        const long long i = ray_i[k] - g.i0, j = ray_j[k] - g.j0;
        if (i < 0 || j < 0 || i >= g.ni || j >= g.nj) return fail(MM_EINVAL, "ray outside the shot grid");
        const unsigned long long t =
            (unsigned long long)(j / kTileY) * (unsigned long long)g.tiles_x + (unsigned long long)(i / kTileX);
        const unsigned long long loc = (unsigned long long)((i % kTileX) + kTileX * (j % kTileY));
        key[(size_t)k] = {t * (unsigned long long)kTileRays + loc, (int)k};
    }
    std::sort(key.begin(), key.end());
    std::vector<unsigned long long> items;
    std::vector<int> begin, local((size_t)n), slot((size_t)n);
    for (int64_t q = 0; q < n; ++q) {
        const unsigned long long t = key[(size_t)q].first / kTileRays;
        if (q == 0 || t != key[(size_t)q - 1].first / kTileRays) {
            items.push_back(t);
            begin.push_back((int)q);
        }
        local[(size_t)q] = (int)(key[(size_t)q].first % kTileRays);
        slot[(size_t)q] = key[(size_t)q].second;
    }
    begin.push_back((int)n);
    // device staging (temporary; returned to the arena's cache)
    struct Tmp {
        DeviceArena *a;
        std::vector<void *> v;
        ~Tmp() { for (void *p : v) a->free(p); }
    } tmp{&ctx->arena, {}};
    auto dalloc = [&](size_t bytes, void **out) -> int {
        int r = ctx->arena.alloc(bytes, out);
        if (!r) tmp.v.push_back(*out);
        return r;
    };
    DumpArgs d{};
    unsigned long long *d_tile;
    int *d_begin, *d_local, *d_slot;
    double *d_alpha;
    long long *d_pixel;
    if ((rc = dalloc(items.size() * 8, (void **)&d_tile)) || (rc = dalloc(begin.size() * 4, (void **)&d_begin)) ||
        (rc = dalloc((size_t)n * 4, (void **)&d_local)) || (rc = dalloc((size_t)n * 4, (void **)&d_slot)) ||
        (rc = dalloc((size_t)n * 16, (void **)&d_alpha)) || (rc = dalloc((size_t)n * 8, (void **)&d_pixel)))
        return rc;
    cudaStream_t s = ctx->stream;
    MM_CUDA(cudaMemcpyAsync(d_tile, items.data(), items.size() * 8, cudaMemcpyHostToDevice, s));
    MM_CUDA(cudaMemcpyAsync(d_begin, begin.data(), begin.size() * 4, cudaMemcpyHostToDevice, s));
    MM_CUDA(cudaMemcpyAsync(d_local, local.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    MM_CUDA(cudaMemcpyAsync(d_slot, slot.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    d.tile = d_tile; d.begin = d_begin; d.local = d_local; d.slot = d_slot; d.alpha = d_alpha; d.pixel = d_pixel;
    ctx->last_launches = 0;
    std::vector<MapObj *> group{M.get()};
    float ms = 0.f;
    rc = launch_group(ctx, group, p->precision, &d, items.size(), s, &ms);
    if (rc) return rc;
    if (alpha_out) MM_CUDA(cudaMemcpyAsync(alpha_out, d_alpha, (size_t)n * 16, cudaMemcpyDeviceToHost, s));
    if (pixel_out) MM_CUDA(cudaMemcpyAsync(pixel_out, d_pixel, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    MM_CUDA(cudaStreamSynchronize(s));
    return MM_OK;
}

int mm_set_variant(mm_ctx *ctx, int32_t variant)
{
    if (!ctx || variant < -1 || variant >= kNumVariants) return fail(MM_EINVAL, "bad variant");
    ctx->forced_variant = variant;
    return MM_OK;
}

int mm_variant_count(void) { return kNumVariants; }

const char *mm_variant_name(int32_t variant) { return variant_name(variant); }

int mm_autotune(mm_ctx *ctx, const mm_params *p, int32_t *variant)
{
    NvtxRange nvtx_("mm_autotune");
    if (!ctx || !p) return fail(MM_EINVAL, "null argument");
    Geo g;
    int rc = compute_geo(p, &g);
    if (rc) return rc;
    cudaSetDevice(ctx->device);
    // a window of the map about 600 tiles large around the grid centre
    mm_params q = *p;
    q.precision = MM_FP32C;
    const long long wi = std::min(g.nx, 64LL * 40), wj = std::min(g.ny, 32LL * 15);
    q.ray_rect[0] = (g.nx - wi) / 2; q.ray_rect[1] = q.ray_rect[0] + wi;
    q.ray_rect[2] = (g.ny - wj) / 2; q.ray_rect[3] = q.ray_rect[2] + wj;
    std::shared_ptr<LensSet> L;
    if ((rc = make_lenses_from_params(ctx, &q, g, ctx->stream, &L))) return rc;
    const int saved_v = ctx->forced_variant, saved_l = ctx->layout;
    double best = 1e300;
    int best_v = 0, best_l = saved_l;
    for (int lay = 0; lay < kNumLayouts && !rc; ++lay) {
        for (int v = 0; v < kNumVariants && !rc; ++v) {
            ctx->forced_variant = v;
            ctx->layout = lay;
            double t_min = 1e300;
            for (int rep = 0; rep < 3; ++rep) {
                std::shared_ptr<MapObj> M;
                Geo gq;
                if ((rc = compute_geo(&q, &gq))) break;
                gq.nstar = L->n;
                if ((rc = alloc_map(ctx, &q, gq, L, ctx->stream, &M))) break;
                std::vector<MapObj *> group{M.get()};
                float ms = 0.f;
                if ((rc = launch_group(ctx, group, false, nullptr, 0, ctx->stream, &ms))) break;
                t_min = std::min(t_min, (double)ms);
            }
            if (t_min < best) { best = t_min; best_v = v; best_l = lay; }
        }
    }
    ctx->forced_variant = saved_v;
    ctx->layout = rc ? saved_l : best_l;
    if (rc) return rc;
    ctx->tuned[class_key(L->unit_mass, L->n)] = best_v;
    if (variant) *variant = best_v;
    return MM_OK;
}

int mm_set_layout(mm_ctx *ctx, int32_t layout)
{
    if (!ctx || layout < 0 || layout >= kNumLayouts) return fail(MM_EINVAL, "bad layout");
    if (ctx->server) return fail(MM_EBUSY, "the layout is fixed once serving has started");
    ctx->layout = layout;
    return MM_OK;
}

int mm_get_layout(mm_ctx *ctx, int32_t *layout)
{
    if (!ctx || !layout) return fail(MM_EINVAL, "null argument");
    *layout = ctx->layout;
    return MM_OK;
}

int mm_layout_count(void) { return kNumLayouts; }

const char *mm_layout_name(int32_t layout) { return layout_name(layout); }

int mm_last_kernel_ms(mm_ctx *ctx, double *ms, int32_t *launches)
{
    if (!ctx) return fail(MM_EINVAL, "null context");
    if (ms) *ms = ctx->last_ms;
    if (launches) *launches = ctx->last_launches;
    return MM_OK;
}

}  // extern "C"
