// mm_internal.h -- structures shared by the host runtime and the device kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mm {

// Ray tile of one CTA: 64 columns x 32 rows of the global ray lattice. Thread t
// owns column (t/32 % 2)*32 + t%32 and the 8 consecutive rows starting at
// (t/64)*8, so the x-differences to a lens are shared by its 8 rays.
constexpr int kThreads = 256;
constexpr int kRaysPerThread = 8;
constexpr int kTileX = 64;
constexpr int kTileY = 32;
constexpr int kTileRays = kTileX * kTileY;
// Lenses are staged into shared memory in chunks of 512 (256 pairs, one per thread).
constexpr int kChunkPairs = 256;
constexpr int kChunkLenses = 2 * kChunkPairs;
// A "null" lens: far enough to contribute < 1e-13 per component, near enough that
// products of two squared distances stay normal in FP32.
constexpr float kNullX = 1.0e13f;
// Lenses within this distance (Einstein radii) of a tile's ray box are summed in FP64.
constexpr float kNearRadius = 0.1f;
// Variants of the FP32 tile computation, chosen per map: (shared-reciprocal pairs per
// 4 lens pairs, fold interval). They differ in rounding, within the accuracy target.
constexpr int kNumVariants = 4;
// Variant of a map without a tuned entry: 0 (3 of 4 pairs share) for unit masses, 2 (2 of
// 4) with masses, where a shared pair also pays two mass products per ray (on GB300 a
// batch of 64 lognormal-mass maps ran at 4.89e12 interactions/s with 2, 4.78e12 with 0).
__host__ __device__ constexpr int default_variant(bool unit_mass) { return unit_mass ? 0 : 2; }
// Thread layouts of the FP32 kernel, chosen per launch: (columns x rows of the 64 x 32
// tile per thread). They give bit-identical maps.
constexpr int kNumLayouts = 4;

// One map of a launch. Built on the host (FP64 geometry), read by the kernels.
struct MapDesc {
    // lattice
    double delta;              // ray spacing
    double half_nx, half_ny;   // nx/2, ny/2
    long long nx, ny;          // global grid
    long long i0, j0, ni, nj;  // shot sub-rectangle [i0, i0+ni) x [j0, j0+nj)
    long long tiles_x;         // ceil(ni / 64)
    // work items: tiles x lens segments; item w = tile * lens_splits + segment
    unsigned long long item_begin;   // first work item of this map in the launch
    unsigned long long item_count;   // work items of this map in the launch
    unsigned long long item_first;   // map work item of the launch's first item (waves)
    int lens_splits;                 // segments per tile (1: whole lens set in one CTA)
    long long seg_lenses;            // lenses per segment, a multiple of kChunkLenses
    // plain FP64 lens equation (FP64 kernel and near-lens terms)
    double one_m_gamma, one_p_gamma, sigma_c, half_side, pix;
    // float-float epilogue: u = A*(2i+1-nx) + N/2 + S/p, S = sum m (x_l - x)/r^2 = -alpha
    float ax_h, ax_l, ay_h, ay_l;   // A_x = (1-gamma-sigma_c) delta / (2p), A_y with 1+gamma
    float ip_h, ip_l;               // 1/p
    float half_n;                   // N_side / 2
    float delta_f, delta_l;         // delta as float-float (ray offsets in a tile)
    int nside;
    int unit_mass;
    int variant;
    int precision;
    long long nstar;
    // lens set (device)
    const double *lx, *ly, *lm;     // FP64 master copy [nstar]
    const float4 *lh;               // (x_hi, y_hi, x_lo, y_lo) padded to a multiple of 512
    const float *lmf;               // FP32 masses, padded (0 for padding)
    // outputs (device)
    unsigned int *counts;           // nside^2
    unsigned long long *totals;     // [0] rays in, [1] rays out (shot is ni*nj)
    // split tiles (lens_splits > 1): per (tile, segment) the float-float sums of the
    // tile's rays, [(tile * lens_splits + segment) * kTileRays + local ray], and per
    // tile the number of segments finished
    float4 *partial;
    unsigned int *seg_done;
    // ray positions: 0 the lattice's cell centres, 1 random in the ray's 64 x 32-cell tile
    // (SplitMix64(ray_seed) outputs 2q + 1, 2q + 2 of ray q = j nx + i)
    int random_rays;
    unsigned long long ray_seed;
};

// Lens segments per tile of a map: split the lens set when a map has too few tiles to
// fill the GPU, so that its work spreads over more CTAs. Depends only on the map.
constexpr unsigned long long kSplitTargetItems = 2048;

// Debug dump: per requested ray, the tile it belongs to and its slot.
struct DumpArgs {
    const unsigned long long *tile;   // per dump tile: tile index within map 0 (work items = tiles x splits)
    const int *begin;                 // per work item: first request [n_items + 1]
    const int *local;                 // per request: local ray index iloc + 64 * jloc, ascending per item
    const int *slot;                  // per request: output slot
    double *alpha;                    // [2 * n_req]
    long long *pixel;                 // [n_req]
};

// Per-launch header in device memory, so that a captured graph can be replayed
// with new work (the host rewrites header + descriptors before each replay).
struct WorkHeader {
    unsigned long long total_work;        // tiles over all maps, or dump work items
    int n_maps;
    int pad;
};

struct LaunchArgs {
    const WorkHeader *hdr;
    const MapDesc *maps;                  // hdr->n_maps descriptors, item_begin ascending
    unsigned long long *work_counter;     // zeroed before the launch
    DumpArgs dump;
    unsigned int *check;                  // checked builds (MM_CHECKS): code of the first failed
                                          // bounds check, zeroed before the launch; else unused
};

// Padded length of a lens set's FP32 tile copies (whole chunks plus one null chunk).
__host__ __device__ inline long long lens_padded(long long nstar)
{
    return (nstar + kChunkLenses - 1) / kChunkLenses * kChunkLenses + kChunkLenses;
}

// ---- launch wrappers (mm_kernels.cu) --------------------------------------
// Build the FP32 tile copies of a lens set: lh[k] = split of (x[k], y[k]) for
// k < n, null lenses for n <= k < n_pad; lmf likewise. n_pad % 512 == 0.
cudaError_t launch_prepare_lenses(const double *x, const double *y, const double *m, long long n,
                                  long long n_pad, float4 *lh, float *lmf, cudaStream_t s);
// Plain FP64 deflection and pixel of n listed rays (global lattice indices ri[k], rj[k])
// of map M, one thread per ray, with the FP64 map kernel's per-ray arithmetic:
// alpha[2k..2k+1], pixel[k] (-1: out or on a lens). Device arrays.
cudaError_t launch_rays_fp64(const MapDesc &M, const long long *ri, const long long *rj, long long n, double *alpha,
                             long long *pixel, cudaStream_t s);
// FP32 (compensated) shoot over the work of args (every map precision MM_FP32C) with
// thread layout `layout`; grid = number of CTAs (persistent); split: some map of the
// launch has lens-split tiles.
cudaError_t launch_shoot_fp32(const LaunchArgs &args, int layout, int grid, bool dump, bool split, cudaStream_t s);
// The FP32 kernel for maps of random rays (MapDesc::random_rays), in thread layout kRandomLayout.
constexpr int kRandomLayout = 3;
cudaError_t launch_shoot_fp32_random(const LaunchArgs &args, int grid, bool dump, bool split, cudaStream_t s);
// Plain FP64 shoot (every map precision MM_FP64).
cudaError_t launch_shoot_fp64(const LaunchArgs &args, int grid, bool dump, cudaStream_t s);
// CTAs per SM the kernels are compiled for (FP32: per thread layout).
int shoot_ctas_per_sm(bool fp64, int layout);
int layout_threads(int layout);
const char *layout_name(int layout);
const char *variant_name(int v);

}  // namespace mm
