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

// Grouped far lenses (far_group_order K > 0): the lens tree of mm_tree.cu.
constexpr int kTreeLevels = 16;           // deepest level of the lens tree
constexpr int kGroupMaxOrder = 32;        // K <= 32 (one moment per lane)
constexpr int kGroupMaxSeries = 16;       // P <= 16 when grouping
constexpr int kBinomN = 64;               // binomial table C(n, k), n, k < 64

// Device view of a lens tree (structure of arrays; node 0 is the root).
struct TreeView {
    double r0;                            // half-side of the root cell
    int K;                                // moments per node
    const unsigned char *level;
    const int *ix, *iy;                   // cell indices at the node's level
    const int *begin, *end;               // the node's lenses: perm[begin .. end)
    const int *first_child, *nchild;      // children first_child .. + nchild (leaf: nchild == 0)
    const double2 *centre;                // z_C
    const double *rc;                     // half-diagonal r_C
    const double *mass;                   // M_C
    const double2 *mom;                   // [node * K + k] = a_k
    const int *perm;                      // lens indices in Morton order
    const double *binom;                  // [n * kBinomN + k] = C(n, k)
};

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
    // grouped far lenses (group > 0): the lens tree and the decisions' FP64 radii
    int group;                            // K (0: every far lens alone)
    double theta;                         // a cell is grouped when rho + r_C <= theta |z_C - z_B|
    double rho64, rn64;                   // block radius and near radius rho / q in FP64
    TreeView tree;
    int *stack;                           // per setup warp: kGroupStack node indices
    unsigned int *overflow;               // set when a setup warp's stack would overflow
    // work items of the production launch: groups of rows_per_item tile rows of a block
    int rows_per_item;                    // 1 or bt
    unsigned long long items;             // nblocks * bt / rows_per_item
    unsigned long long item_begin;        // first launch item of this map
    unsigned long long item_first;        // the map item of that launch item (serving waves)
};

constexpr int kGroupStack = 4096;         // stack entries per setup warp

// Grouped setup of every block (F.group > 0), one warp per block: with near_idx == nullptr the
// near-lens counts into a[b], the series coefficients and the bounds; else the near lenses of
// every block from F.near_off[b] on (the same walk, so the same order).
cudaError_t launch_far_group(const MapDesc &M, const FarDesc &F, float *coef, unsigned long long *a, int *near_idx,
                             int warps, cudaStream_t s);
int far_group_warps(int sms);

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
