// mm_device.cuh -- device helpers shared by the shooting kernels (one copy per
// translation unit): float-float arithmetic, shared-memory layout, the
// persistent work loop and the debug-dump lookup.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "mm_internal.h"

// Checked builds (-DMM_CHECKS): a failed bounds check records its site code in
// *check (the first failure wins) and the guarded access is skipped, so that a
// bad index becomes a status the host reads instead of a fault. Other builds
// compile the checks away.
#ifdef MM_CHECKS
#define MM_BOUNDS(check, cond, code) \
    ((cond) ? true : (atomicCAS((check), 0u, (unsigned)(code)), false))
#else
#define MM_BOUNDS(check, cond, code) true
#endif

namespace mm {
namespace dev {

// Site codes of the bounds checks.
enum CheckSite : unsigned {
    kChkMapCount = 1,       // a count outside the N_side^2 map
    kChkLensTile = 2,       // an FP32 lens tile read past the padded lens set
    kChkLensFP64 = 3,       // an FP64 lens read past N*
    kChkPartial = 4,        // a split tile's partial sums outside its buffer
    kChkSegDone = 5,        // a split tile's segment counter outside its buffer
    kChkNearList = 6,       // a far-field near-list access outside the list
    kChkFarBlock = 7,       // a far-field block index outside the map's blocks
};

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Error-free transformation a + b = s + e (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Add an FP64 value into a float-float accumulator (h, l).
__device__ __forceinline__ void add_ff(float &h, float &l, double v)
{
    const float vh = __double2float_rn(v);
    const float vl = __double2float_rn(v - (double)vh);
    float s, e;
    two_sum(h, vh, s, e);
    h = s;
    l = __fadd_rn(l, __fadd_rn(e, vl));
}

// Float-float u = (ch + cl) * n + base for an exactly representable integer-valued n.
__device__ __forceinline__ void ff_axis(float ch, float cl, float n, float base, float &uh, float &ul)
{
    const float ph = __fmul_rn(ch, n);
    float pe = __fmaf_rn(ch, n, -ph);
    pe = __fmaf_rn(cl, n, pe);
    float s, e;
    two_sum(base, ph, s, e);
    uh = s;
    ul = __fadd_rn(e, pe);
}

// floor(u) for u = (uh + ul) + (sh + sl) * (iph + ipl), evaluated in float-float.
__device__ __forceinline__ float ff_pixel(float uh, float ul, float sh, float sl, float iph, float ipl)
{
    const float th = __fmul_rn(sh, iph);
    float te = __fmaf_rn(sh, iph, -th);
    te = __fmaf_rn(sh, ipl, te);
    te = __fmaf_rn(sl, iph, te);
    float s, e;
    two_sum(uh, th, s, e);
    const float lo = __fadd_rn(__fadd_rn(e, ul), te);
    const float I = floorf(s);
    const float f = __fadd_rn(__fsub_rn(s, I), lo);
    return __fadd_rn(I, floorf(f));
}

// Float-float u = (ch + cl) * (n + f) + base for an exactly representable integer-valued n and an
// exactly representable f (the offset of a random ray within its tile, in half cells).
__device__ __forceinline__ void ff_axis_frac(float ch, float cl, float n, float f, float base, float &uh, float &ul)
{
    ff_axis(ch, cl, n, base, uh, ul);
    const float ph = __fmul_rn(ch, f);
    float pe = __fmaf_rn(ch, f, -ph);
    pe = __fmaf_rn(cl, f, pe);
    float s, e;
    two_sum(uh, ph, s, e);
    uh = s;
    ul = __fadd_rn(ul, __fadd_rn(e, pe));
}

// Random rays (MapDesc::random_rays), as the paper's GPU code shoots them (Sect. 2.3, step 2):
// output k >= 1 of SplitMix64 seeded with s (Steele, Lea & Flood, OOPSLA 2014) is
// mix(s + k * 0x9E3779B97F4A7C15 mod 2^64), mix the generator's finaliser.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long s, unsigned long long k)
{
    unsigned long long z = s + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Random ray (gi, gj) lies at (fx, fy) cells from the corner of its 64 x 32-cell tile: fx = u1 wi,
// fy = u2 wj, u1 and u2 the top 18 bits of outputs 2q + 1 and 2q + 2 (q = gj nx + gi) as fractions,
// wi and wj the tile's width and height in cells (partial at the grid's far edges). Both are exact in
// single precision (at most 24 significant bits).
__device__ __forceinline__ void random_cell(const MapDesc &M, long long gi, long long gj, float &fx, float &fy)
{
    const unsigned long long q = (unsigned long long)gj * (unsigned long long)M.nx + (unsigned long long)gi;
    const unsigned u1 = (unsigned)(splitmix64_at(M.ray_seed, 2 * q + 1) >> 46);
    const unsigned u2 = (unsigned)(splitmix64_at(M.ray_seed, 2 * q + 2) >> 46);
    const long long ti = gi / kTileX, tj = gj / kTileY;
    const unsigned wi = (unsigned)min((long long)kTileX, M.nx - kTileX * ti);
    const unsigned wj = (unsigned)min((long long)kTileY, M.ny - kTileY * tj);
    fx = (float)(u1 * wi) * (1.0f / 262144.0f);
    fy = (float)(u2 * wj) * (1.0f / 262144.0f);
}

// FP64 coordinate of a random ray along one axis: (t0 + f - n/2) delta, t0 its tile's first cell.
__device__ __forceinline__ double random_coord(long long t0, float f, double half_n, double delta)
{
    return __dmul_rn(__dsub_rn(__dadd_rn((double)t0, (double)f), half_n), delta);
}

// Shared state of the persistent loop (first member of each kernel's shared block).
struct LoopSmem {
    unsigned long long g;          // the next work item (fetched ahead) and its map
    int map;
    unsigned red_in, red_out;
    int last_segment;              // split tiles: this CTA finished the tile's last segment
};

// Float-float addition of two (x_hi, x_lo, y_hi, y_lo) sums (lo parts unnormalised).
__device__ __forceinline__ float4 ff_add4(float4 a, float4 b)
{
    float s, e;
    two_sum(a.x, b.x, s, e);
    a.x = s;
    a.y = __fadd_rn(a.y, __fadd_rn(e, b.y));
    two_sum(a.z, b.z, s, e);
    a.z = s;
    a.w = __fadd_rn(a.w, __fadd_rn(e, b.w));
    return a;
}

struct __align__(16) SmemFP32 {
    float4 pos[kChunkPairs];       // (xa, xb, ya, yb) relative to the tile centre
    float2 mass[kChunkPairs];      // (ma, mb)
    float4 acc[kTileRays];         // per ray: float-float sums (x_hi, x_lo, y_hi, y_lo), [slot][thread]
    unsigned near_bits[2 * kChunkPairs / 32];
    double cx, cy;                 // tile centre (FP64)
    LoopSmem loop;
};

struct __align__(16) SmemFP64 {
    double2 lens64[kChunkPairs];   // (x, y) of lens k of the chunk
    double m64[kChunkPairs];
    LoopSmem loop;
};

__device__ __forceinline__ int find_map(const LaunchArgs &A, int n_maps, unsigned long long g)
{
    int lo = 0, hi = n_maps - 1;
    while (lo < hi) {                              // last map with item_begin <= g
        const int mid = (lo + hi + 1) >> 1;
        if (A.maps[mid].item_begin <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// First request of work item `item` with local ray index `mine` (requests of an item
// are sorted by local index), or -1.
__device__ __forceinline__ int dump_find(const DumpArgs &D, int item, int mine)
{
    int lo = D.begin[item], hi = D.begin[item + 1];
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (D.local[mid] < mine) lo = mid + 1; else hi = mid;
    }
    return (lo < D.begin[item + 1] && D.local[lo] == mine) ? lo : -1;
}

// Record one ray's result: debug dump, or a warp-aggregated count into the map
// (every lane of the warp must call this together, lanes in column order).
template <bool DUMP>
__device__ __forceinline__ void emit_ray(const LaunchArgs &A, const MapDesc &M, int item, int local, bool valid,
                                         bool inside, unsigned pix, double alpha1, double alpha2, unsigned &cnt_in,
                                         unsigned &cnt_out)
{
    if (DUMP) {
        for (int q = dump_find(A.dump, item, local); q >= 0 && q < A.dump.begin[item + 1] && A.dump.local[q] == local;
             ++q) {
            const int sl = A.dump.slot[q];
            A.dump.alpha[2 * sl] = alpha1;
            A.dump.alpha[2 * sl + 1] = alpha2;
            A.dump.pixel[sl] = inside ? (long long)pix : -1LL;
        }
    } else {
        // The lanes of a warp hold consecutive columns of one lattice row, so rays that
        // land in the same pixel come in runs: the first lane of each run adds its length.
        const unsigned lane = threadIdx.x & 31;
        const unsigned key = inside ? pix : 0xffffffffu;
        const unsigned left = __shfl_up_sync(0xffffffffu, key, 1);
        const bool start = lane == 0 || left != key;
        const unsigned starts = __ballot_sync(0xffffffffu, start);
        if (inside && start && MM_BOUNDS(A.check, pix < (unsigned)M.nside * (unsigned)M.nside, kChkMapCount)) {
            const unsigned above = starts & ~((2u << lane) - 1u);     // run starts after this lane
            atomicAdd(M.counts + pix, (above ? (unsigned)(__ffs(above) - 1) : 32u) - lane);
        }
        cnt_in += inside ? 1u : 0u;
        cnt_out += (valid && !inside) ? 1u : 0u;
    }
}

// Persistent loop: take work items from the launch's counter until exhausted,
// run `body(M, tile, segment, dump_item, cnt_in, cnt_out)` on each, and add the
// in/out ray counts to the map totals whenever the map changes and at exit. The
// next item is fetched while the current one runs, so the counter's latency is
// hidden behind the work.
template <bool DUMP, typename Body>
__device__ __forceinline__ void persistent_loop(const LaunchArgs &A, LoopSmem &S, Body body)
{
    const int tid = threadIdx.x;
    int cur_map = -1;
    unsigned long long run_in = 0, run_out = 0;   // meaningful in thread 0
    const unsigned long long total_work = A.hdr->total_work;
    const int n_maps = A.hdr->n_maps;
    if (tid == 0) {
        const unsigned long long g = atomicAdd(A.work_counter, 1ULL);
        S.g = g;
        S.map = (g < total_work) ? (DUMP ? 0 : find_map(A, n_maps, g)) : -1;
        S.red_in = 0;
        S.red_out = 0;
    }
    __syncthreads();
    for (;;) {
        const unsigned long long g = S.g;
        const int mi = S.map;
        if (g >= total_work) break;
        __syncthreads();                           // every thread has read S.g and S.map
        if (tid == 0) {
            const unsigned long long gn = atomicAdd(A.work_counter, 1ULL);   // the next item, ahead
            S.g = gn;
            S.map = (gn < total_work) ? (DUMP ? 0 : find_map(A, n_maps, gn)) : -1;
            if (cur_map != mi) {
                if (cur_map >= 0 && !DUMP) {
                    atomicAdd(A.maps[cur_map].totals + 0, run_in);
                    atomicAdd(A.maps[cur_map].totals + 1, run_out);
                }
                cur_map = mi;
                run_in = run_out = 0;
            }
        }
        const MapDesc &M = A.maps[mi];
        const unsigned long long nsp = (unsigned long long)M.lens_splits;
        const unsigned long long work =
            DUMP ? A.dump.tile[g / nsp] * nsp + g % nsp : M.item_first + (g - M.item_begin);
        unsigned ci = 0, co = 0;
        body(M, work / nsp, (int)(work % nsp), DUMP ? (int)(g / nsp) : 0, ci, co);
        if (!DUMP) {
            ci = __reduce_add_sync(0xffffffffu, ci);
            co = __reduce_add_sync(0xffffffffu, co);
            if ((tid & 31) == 0) {
                atomicAdd(&S.red_in, ci);
                atomicAdd(&S.red_out, co);
            }
        }
        __syncthreads();
        if (tid == 0) {
            run_in += S.red_in;
            run_out += S.red_out;
            S.red_in = 0;                          // for the next item (its body may hold no barrier)
            S.red_out = 0;
        }
        __syncthreads();                           // S.g, S.map and S.red_* are ready for the next item
    }
    if (tid == 0 && cur_map >= 0 && !DUMP) {
        atomicAdd(A.maps[cur_map].totals + 0, run_in);
        atomicAdd(A.maps[cur_map].totals + 1, run_out);
    }
}

}  // namespace dev
}  // namespace mm
