// mm_far.h -- far-field approximation (MM_FAR32): the tree code's idea (Sect. 2.1,
// Eq. hierarchical) on blocks of rays. Shared by the host runtime and mm_far.cu.
//
// The ray lattice of a map is cut into blocks of bt x bt tiles (64 bt x 32 bt rays),
// counted from the shot rectangle's origin. For block B with centre z_B and radius
// rho (half-diagonal of its lattice cells), every lens with |z_i - z_B| < rho / q
// is "near" and summed exactly for each ray of B; the others enter
//     sum_far m_i / (z - z_i) = sum_{l<P} c'_l v^l,   v = (z - z_B) / rho,
//     c'_l = -rho^l sum_far m_i / d_i^(l+1),           d_i = z_i - z_B,
// and conj() of that sum is their deflection (alpha = conj(sum m / (z - z_i))).
// The series in v keeps every coefficient below sum m / |d| q^l, so no power
// overflows FP32 whatever the block size.
#pragma once
#include <cuda_runtime.h>

#include "mm_internal.h"

namespace mm {

constexpr int kFarMaxOrder = 32;
constexpr int kFarMaxBlock = 64;
constexpr int kFarThreads = 256;

// Far-field description of one MM_FAR32 map of a launch (parallel to its MapDesc).
struct FarDesc {
    int order;                            // series terms P
    int bt;                               // block side in tiles
    long long blocks_x, blocks_y, nblocks;
    int stride;                           // floats per block in coef (a multiple of 4)
    float rn2;                            // (rho / q)^2, compared with FP32 squared offsets
    float rho;                            // block radius
    float dv_h, dv_l;                     // Delta / rho as float-float (ray offsets in v)
    const float *coef;                    // per block: c'_0 as (re_h, re_l, im_h, im_l), then
                                          // (re, im) of c'_l for l = 1 .. P-1
    const unsigned long long *near_off;   // [nblocks + 1]: near lenses of block b are
                                          // near_idx[near_off[b] .. near_off[b + 1])
    const int *near_idx;                  // ascending lens indices per block
    unsigned int *bound_max;              // bits of the largest block bound (a positive float)
    unsigned int *check;                  // checked builds: first failed bounds check (see LaunchArgs)
    // work items of the production launch: groups of rows_per_item tile rows of a block
    int rows_per_item;                    // 1 or bt
    unsigned long long items;             // nblocks * bt / rows_per_item
    unsigned long long item_begin;        // first launch item of this map
    unsigned long long item_first;        // the map item of that launch item (serving waves)
};

// Near-lens count of every block into a[b] (b < F.nblocks).
cudaError_t launch_far_count(const MapDesc &M, const FarDesc &F, unsigned long long *a, int grid, cudaStream_t s);
// In-place exclusive prefix sum of a[0 .. n); a[n] receives the total.
cudaError_t launch_far_scan(unsigned long long *a, long long n, cudaStream_t s);
// Series coefficients, near lists and bounds of every block (F.near_off must be final).
cudaError_t launch_far_setup(const MapDesc &M, const FarDesc &F, float *coef, int *near_idx, int grid,
                             cudaStream_t s);
// Persistent shoot (every map MM_FAR32; far[k] describes args.maps[k]) over total_items
// work items (FarDesc::items summed over the maps), or, with dump, over the dump's tiles.
cudaError_t launch_shoot_far(const LaunchArgs &args, const FarDesc *far, unsigned long long total_items, int grid,
                             bool dump, cudaStream_t s);
int far_ctas_per_sm();

}  // namespace mm
