// mm_far.cu -- the far-field approximation MM_FAR32 (see mm_far.h): the tree code's
// idea of Sect. 2.1 (Eq. hierarchical: near lenses one by one, distant ones grouped;
// pseudo-lens deflections computed at test rays and interpolated for the rays around
// them), recast for the GPU. The test ray is the centre of a block of ray tiles; the
// "interpolation" is the series of the far lenses' deflection about it, with a
// rigorous tail bound instead of an empirical accuracy.
//
// Per map, before its rays are shot:
//   k_far_count  near-lens count of every block, one warp per block (FP32 offsets,
//                explicit rounding, so that every kernel decides alike);
//   k_far_scan   exclusive prefix sum of the counts (near-list offsets);
//   k_far_fill   the near lenses of every block in index order, one warp per block;
//   k_far_setup  per block: the series coefficients c'_0 (float-float) and c'_l
//                (FP32), l < P, and the tail bound.
// Then the persistent k_shoot_far takes work items of whole blocks (or single tile
// rows of a block, when a map has few blocks): the block's series and near lenses
// are staged in shared memory once, and its 64 x 32-ray tiles follow without a
// barrier. Each ray evaluates the series by Horner's rule in v = (z - z_B) / rho
// (packed f32x2 over pairs of rows) and adds its block's near lenses: FP32 terms
// relative to the tile centre, FP64 terms for lenses within kNearRadius of the
// tile's ray box. The float-float lens equation is the exact FP32 kernel's; the
// count goes to the map by run-length warp aggregation (rays of a warp share a
// lattice row, so equal pixels come in runs). The debug dump runs the same tile
// code one tile at a time.
#include <algorithm>
#include <cmath>
#include <vector>

#include "mm_ctx.h"
#include "mm_device.cuh"
#include "mm_far.h"

namespace mm {
namespace dev {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kFarWarps = kFarThreads / 32;
constexpr int kShootThreads = 256;                 // threads of the shoot kernels' CTAs (2 per SM)
constexpr int kFarRows = kTileRays / kShootThreads; // rays per thread: one column, 8 rows

__device__ __forceinline__ void split_d(double v, float &h, float &l)
{
    h = __double2float_rn(v);
    l = __double2float_rn(v - (double)h);
}

// Centre of block (bx, by) of map M (FP64).
__device__ __forceinline__ void far_centre(const MapDesc &M, const FarDesc &F, long long bx, long long by,
                                           double &xb, double &yb)
{
    const long long bw = 64LL * F.bt, bh = 32LL * F.bt;
    xb = ((double)(M.i0 + bx * bw + bw / 2) - M.half_nx) * M.delta;
    yb = ((double)(M.j0 + by * bh + bh / 2) - M.half_ny) * M.delta;
}

// Offset of a lens (float-float coordinates q) from a float-float centre, and its
// squared length, rounded step by step, so that every kernel takes the same near
// decision for the same lens and block.
__device__ __forceinline__ void far_offset(const float4 q, float cxh, float cxl, float cyh, float cyl, float &dx,
                                           float &dy, float &r2)
{
    dx = __fadd_rn(__fsub_rn(q.x, cxh), __fsub_rn(q.z, cxl));
    dy = __fadd_rn(__fsub_rn(q.y, cyh), __fsub_rn(q.w, cyl));
    r2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

// One warp per block: the near-lens count of block b into a[b].
__global__ void __launch_bounds__(kFarThreads) k_far_count(const MapDesc M, const FarDesc F, unsigned long long *a)
{
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * kFarWarps;
    for (long long b = (long long)blockIdx.x * kFarWarps + (threadIdx.x >> 5); b < F.nblocks; b += warps) {
        double xb, yb;
        far_centre(M, F, b % F.blocks_x, b / F.blocks_x, xb, yb);
        float cxh, cxl, cyh, cyl;
        split_d(xb, cxh, cxl);
        split_d(yb, cyh, cyl);
        unsigned cnt = 0;
        for (long long k = lane; k < M.nstar; k += 32) {
            float dx, dy, r2;
            far_offset(M.lh[k], cxh, cxl, cyh, cyl, dx, dy, r2);
            cnt += r2 < F.rn2 ? 1u : 0u;
        }
        cnt = __reduce_add_sync(kFull, cnt);
        if (lane == 0) a[b] = cnt;
    }
}

// One warp per block: the near lenses of block b, in index order, from near_off[b].
__global__ void __launch_bounds__(kFarThreads) k_far_fill(const MapDesc M, const FarDesc F, int *near_idx)
{
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * kFarWarps;
    for (long long b = (long long)blockIdx.x * kFarWarps + (threadIdx.x >> 5); b < F.nblocks; b += warps) {
        double xb, yb;
        far_centre(M, F, b % F.blocks_x, b / F.blocks_x, xb, yb);
        float cxh, cxl, cyh, cyl;
        split_d(xb, cxh, cxl);
        split_d(yb, cyh, cyl);
        unsigned long long out = F.near_off[b];
        for (long long base = 0; base < M.nstar; base += 32) {
            const long long k = base + lane;
            bool near = false;
            if (k < M.nstar) {
                float dx, dy, r2;
                far_offset(M.lh[k], cxh, cxl, cyh, cyl, dx, dy, r2);
                near = r2 < F.rn2;
            }
            const unsigned bal = __ballot_sync(kFull, near);
            const unsigned long long at = out + __popc(bal & ((1u << lane) - 1u));
            if (near && MM_BOUNDS(F.check, at < F.near_off[b + 1], kChkNearList)) near_idx[at] = (int)k;
            out += __popc(bal);
        }
    }
}

// One CTA of 1024 threads walks the array in chunks, carrying the running total.
__global__ void __launch_bounds__(1024) k_far_scan(unsigned long long *a, long long n)
{
    __shared__ unsigned long long wsum[32];
    __shared__ unsigned long long carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long base = 0; base < n; base += 1024) {
        const long long i = base + threadIdx.x;
        const unsigned long long v = i < n ? a[i] : 0ULL;
        unsigned long long x = v;                             // inclusive scan within the warp
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {                                         // inclusive scan of the warp totals
            unsigned long long t = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(kFull, t, o);
                if (lane >= o) t += y;
            }
            wsum[lane] = t;
        }
        __syncthreads();
        if (i < n) a[i] = carry + (w > 0 ? wsum[w - 1] : 0ULL) + x - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) a[n] = carry;
}

// One CTA per block: the series coefficients of its far lenses and its tail bound at
// |w| = rho (the near lenses are k_far_fill's). PMAX >= F.order.
template <int PMAX, bool MASS>
__global__ void __launch_bounds__(kFarThreads) k_far_setup(const MapDesc M, const FarDesc F, float *coef)
{
    constexpr int NC = PMAX > 1 ? PMAX - 1 : 1;
    __shared__ float red_c[kFarWarps][2 * NC];
    __shared__ float4 red_0[kFarWarps];
    __shared__ float red_b[kFarWarps];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int P = F.order;
    const float rho = F.rho;
    for (long long b = blockIdx.x; b < F.nblocks; b += gridDim.x) {
        double xb, yb;
        far_centre(M, F, b % F.blocks_x, b / F.blocks_x, xb, yb);
        float cxh, cxl, cyh, cyl;
        split_d(xb, cxh, cxl);
        split_d(yb, cyh, cyl);
        float c0rh = 0.f, c0rl = 0.f, c0ih = 0.f, c0il = 0.f;
        float cr[NC], ci[NC];
#pragma unroll
        for (int l = 0; l < NC; ++l) cr[l] = ci[l] = 0.f;
        float bnd = 0.f;
        for (long long k = tid; k < M.nstar; k += kFarThreads) {
            float dx, dy, r2;
            far_offset(M.lh[k], cxh, cxl, cyh, cyl, dx, dy, r2);
            if (!(r2 < F.rn2)) {                              // far (the near lenses are k_far_fill's)
                const float m = MASS ? M.lmf[k] : 1.f;
                const float inv = rcp_approx(r2);
                const float ur = __fmul_rn(dx, inv), ui = -__fmul_rn(dy, inv);   // u = 1 / d
                float tr = -m * ur, ti = -m * ui;                                 // -m / d
                float s, e;
                two_sum(c0rh, tr, s, e);
                c0rh = s;
                c0rl = __fadd_rn(c0rl, e);
                two_sum(c0ih, ti, s, e);
                c0ih = s;
                c0il = __fadd_rn(c0il, e);
                const float sr = rho * ur, si = rho * ui;                         // rho / d, |rho / d| < q
#pragma unroll
                for (int l = 1; l < PMAX; ++l) {
                    if (l < P) {                                                  // -m rho^l / d^(l+1)
                        const float nr = fmaf(tr, sr, -ti * si);
                        const float ni = fmaf(tr, si, ti * sr);
                        tr = nr;
                        ti = ni;
                        cr[l - 1] += tr;
                        ci[l - 1] += ti;
                    }
                }
                const float dinv = rsqrtf(r2);                                    // 1 / |d|
                const float t = rho * dinv;
                bnd = fmaf(m * dinv, exp2f((float)P * __log2f(t)) / (1.f - t), bnd);
            }
        }
        // CTA reduction: butterfly within warps, then warps in order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float s, e;
            const float rh = __shfl_xor_sync(kFull, c0rh, o), rl = __shfl_xor_sync(kFull, c0rl, o);
            two_sum(c0rh, rh, s, e);
            c0rh = s;
            c0rl = __fadd_rn(__fadd_rn(c0rl, rl), e);
            const float ih = __shfl_xor_sync(kFull, c0ih, o), il = __shfl_xor_sync(kFull, c0il, o);
            two_sum(c0ih, ih, s, e);
            c0ih = s;
            c0il = __fadd_rn(__fadd_rn(c0il, il), e);
#pragma unroll
            for (int l = 0; l < NC; ++l) {
                if (l + 1 < P) {
                    cr[l] += __shfl_xor_sync(kFull, cr[l], o);
                    ci[l] += __shfl_xor_sync(kFull, ci[l], o);
                }
            }
            bnd += __shfl_xor_sync(kFull, bnd, o);
        }
        if (lane == 0) {
            red_0[w] = make_float4(c0rh, c0rl, c0ih, c0il);
#pragma unroll
            for (int l = 0; l < NC; ++l) {
                red_c[w][2 * l] = cr[l];
                red_c[w][2 * l + 1] = ci[l];
            }
            red_b[w] = bnd;
        }
        __syncthreads();
        float *cb = coef + b * (long long)F.stride;
        if (tid == 0) {
            float4 a0 = red_0[0];
            float tb = red_b[0];
            for (int q = 1; q < kFarWarps; ++q) {
                a0 = ff_add4(a0, red_0[q]);
                tb += red_b[q];
            }
            cb[0] = a0.x;
            cb[1] = a0.y;
            cb[2] = a0.z;
            cb[3] = a0.w;
            // a little above the FP32 sum (fast log2 / exp2, rounding), so that the bound stays a bound
            atomicMax(F.bound_max, __float_as_uint(tb * 1.001f));
        }
        for (int c = tid; c < 2 * (P - 1); c += kFarThreads) {
            float v = red_c[0][c];
            for (int q = 1; q < kFarWarps; ++q) v += red_c[q][c];
            cb[4 + c] = v;
        }
        __syncthreads();                                      // red_* are rewritten by the next block
    }
}

constexpr int kNearCap = 512;                 // near lenses staged at once per item
constexpr int kNearFold = 32;                 // near terms summed in FP32 between float-float folds

struct __align__(16) SmemFar {
    float4 nl[kNearCap];                      // near lens offset from the block centre, float-float (xh, xl, yh, yl)
    float nm[kNearCap];                       // its mass
    int ng[kNearCap];                         // its index, for FP64 terms
    float coef[4 + 2 * (kFarMaxOrder - 1)];   // the block's series
    unsigned long long next;                  // next work item (production loop)
    long long chunk0;                         // first near lens held in nl/nm/ng
    LoopSmem loop;                            // debug dump loop
    unsigned red_in, red_out;
};

// Stage the series of block blk and its near lenses [c0, c0 + kNearCap) into shared
// memory (called by all threads; the caller synchronises before and after).
__device__ __forceinline__ void far_stage(const MapDesc &M, const FarDesc &F, long long blk, long long c0, bool coefs,
                                          SmemFar &S)
{
    const int tid = threadIdx.x;
    if (coefs)
        for (int c = tid; c < 4 + 2 * (F.order - 1); c += kShootThreads) S.coef[c] = F.coef[blk * (long long)F.stride + c];
    double xb, yb;
    far_centre(M, F, blk % F.blocks_x, blk / F.blocks_x, xb, yb);
    float cxh, cxl, cyh, cyl;
    split_d(xb, cxh, cxl);
    split_d(yb, cyh, cyl);
    const unsigned long long off0 = F.near_off[blk];
    const long long n_near = (long long)(F.near_off[blk + 1] - off0);
    const long long end = min(n_near, c0 + (long long)kNearCap);
    for (long long k = c0 + tid; k < end; k += kShootThreads) {
        if (!MM_BOUNDS(F.check, off0 + k < F.near_off[F.nblocks], kChkNearList)) continue;
        const int g = F.near_idx[off0 + k];
        if (!MM_BOUNDS(F.check, g >= 0 && g < M.nstar, kChkNearList)) continue;
        const float4 q = M.lh[g];
        float sh, se, th, te;
        two_sum(q.x, -cxh, sh, se);                           // exact split of x_h - c_h
        two_sum(q.y, -cyh, th, te);
        S.nl[k - c0] = make_float4(sh, __fadd_rn(se, __fsub_rn(q.z, cxl)), th, __fadd_rn(te, __fsub_rn(q.w, cyl)));
        S.nm[k - c0] = M.unit_mass ? 1.f : M.lmf[g];
        S.ng[k - c0] = g;
    }
    if (tid == 0) S.chunk0 = c0;
}

// Production binning: rays of a warp lie along one lattice row, so equal pixels
// come in runs; the first lane of each run adds the run's length.
// counts / npix: the map's counts and N_side^2, passed by value: read through the map
// descriptor they would be reloaded after every atomic, which may alias it. The first
// lane of a run also adds the run's length to cnt_in (the production kernel counts the
// valid rays per tile and takes the rays out as the difference).
__device__ __forceinline__ void far_bin(unsigned *counts, unsigned npix, unsigned *check, bool inside, unsigned pix,
                                        unsigned &cnt_in)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned key = inside ? pix : 0xffffffffu;
    const unsigned left = __shfl_up_sync(kFull, key, 1);
    const bool start = lane == 0 || left != key;
    const unsigned starts = __ballot_sync(kFull, start);
    if (inside && start && MM_BOUNDS(check, pix < npix, kChkMapCount)) {
        const unsigned above = starts & ~((2u << lane) - 1u);    // run starts after this lane
        const unsigned run = (above ? (unsigned)(__ffs(above) - 1) : 32u) - lane;
        atomicAdd(counts + pix, run);
        cnt_in += run;
    }
}

// Float-float steps on a pair of rows (f32x2). Lane by lane they round exactly as
// ff_axis / ff_pixel / two_sum do: x - y is formed as fma(y, -1, x) (an exact product,
// one rounding), and the negated products -RN(c n) as RN((-c) n). Only the sign of an
// exact zero may differ, which no pixel index sees.
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

__device__ __forceinline__ float2 sub2(float2 x, float2 y, float2 m1) { return __ffma2_rn(y, m1, x); }

// s = RN(a + b) and its rounding error e, given nb = -b.
__device__ __forceinline__ void two_sum2(float2 a, float2 nb, float2 m1, float2 &s, float2 &e)
{
    s = sub2(a, nb, m1);
    const float2 bb = sub2(s, a, m1);
    const float2 e1 = sub2(a, sub2(s, bb, m1), m1);
    e = sub2(e1, __fadd2_rn(nb, bb), m1);                 // e1 + (b - bb)
}

// u = (ch + cl) n + base in float-float, for two exactly representable n (nch = -ch).
__device__ __forceinline__ void ff_axis2(float2 ch, float2 nch, float2 cl, float2 n, float2 base, float2 m1,
                                         float2 &uh, float2 &ul)
{
    const float2 nph = __fmul2_rn(nch, n);
    float2 pe = __ffma2_rn(ch, n, nph);
    pe = __ffma2_rn(cl, n, pe);
    float2 e;
    two_sum2(base, nph, m1, uh, e);
    ul = __fadd2_rn(e, pe);
}

// floor(u) for u = (uh + ul) + (sh + sl) (iph + ipl), two rays (niph = -iph).
__device__ __forceinline__ float2 ff_pixel2(float2 uh, float2 ul, float2 sh, float2 sl, float2 iph, float2 niph,
                                            float2 ipl, float2 m1)
{
    const float2 nth = __fmul2_rn(sh, niph);
    float2 te = __ffma2_rn(sh, iph, nth);
    te = __ffma2_rn(sh, ipl, te);
    te = __ffma2_rn(sl, iph, te);
    float2 s, e;
    two_sum2(uh, nth, m1, s, e);
    const float2 lo = __fadd2_rn(__fadd2_rn(e, ul), te);
    const float2 I = make_float2(floorf(s.x), floorf(s.y));
    const float2 f = __fadd2_rn(sub2(s, I, m1), lo);
    return __fadd2_rn(I, make_float2(floorf(f.x), floorf(f.y)));
}

__device__ __forceinline__ float &lane(float2 &v, int l) { return l ? v.y : v.x; }

// Pixel bases of a block's rays: u = A (2i + 1 - n) + N/2 + S / p with S = -alpha; the
// block's c'_0 part of S/p is the same for all its rays and enters the bases
// kx = N/2 - Re c'_0 / p, ky = N/2 + Im c'_0 / p (float-float). Needs the block's
// series staged in S.
struct FarBase {
    float kxh, kxl, kyh, kyl;
};

__device__ __forceinline__ FarBase far_base(const MapDesc &M, const SmemFar &S)
{
    const float c0rh = S.coef[0], c0rl = S.coef[1], c0ih = S.coef[2], c0il = S.coef[3];
    FarBase B;
    float ph = __fmul_rn(c0rh, M.ip_h);
    float pe = __fmaf_rn(c0rh, M.ip_h, -ph);
    pe = __fmaf_rn(c0rh, M.ip_l, __fmaf_rn(c0rl, M.ip_h, pe));
    float e;
    two_sum(M.half_n, -ph, B.kxh, e);
    B.kxl = __fsub_rn(e, pe);
    ph = __fmul_rn(c0ih, M.ip_h);
    pe = __fmaf_rn(c0ih, M.ip_h, -ph);
    pe = __fmaf_rn(c0ih, M.ip_l, __fmaf_rn(c0il, M.ip_h, pe));
    two_sum(M.half_n, ph, B.kyh, e);
    B.kyl = __fadd_rn(e, pe);
    return B;
}

// The rays of tile (tx, ty), whose block's series and first near chunk are staged in
// S. Near lists longer than kNearCap are re-staged chunk by chunk (uniform syncs).
template <bool DUMP, bool MASS>
__device__ void far_tile(const LaunchArgs &A, const FarDesc &F, const MapDesc &M, long long blk, long long bx,
                         long long by, const FarBase &B, long long tx, long long ty, int item, SmemFar &S,
                         unsigned &cnt_in, unsigned &cnt_out)
{
    constexpr int K = kFarRows;
    const int tid = threadIdx.x, w = tid >> 5;
    const int iloc = (w & 1) * 32 + (tid & 31);
    const int jloc0 = (w >> 1) * K;
    const long long ib = M.i0 + tx * kTileX, jb = M.j0 + ty * kTileY;
    const long long bw = 64LL * F.bt, bh = 32LL * F.bt;
    const long long ibB = M.i0 + bx * bw, jbB = M.j0 + by * bh;     // block (bx, by) = blk, from the caller
    const int P = F.order;

    // ---- far series: Horner's rule in v = (z - z_B) / rho, packed over row pairs ----
    // Lattice offsets are formed in 32-bit integers (|n| <= bw / 2) and rows by exact
    // float steps: no 64-bit integer conversion per ray.
    const float nxo = (float)(int)(ib + iloc - ibB - bw / 2) + 0.5f;
    const float vx = __fmaf_rn(nxo, F.dv_h, __fmul_rn(nxo, F.dv_l));
    const float nyo0 = (float)(int)(jb + jloc0 - jbB - bh / 2) + 0.5f;
    constexpr int H = K / 2;
    // float-float sums of S = -alpha per row pair (lane l: row 2q + l): x (hi, lo), y (hi, lo)
    float2 SXh[H], SXl[H], SYh[H], SYl[H];
    {
        float2 VY[H], VYN[H], SR[H], SI[H];
#pragma unroll
        for (int q = 0; q < H; ++q) {
            const float na = nyo0 + (float)(2 * q), nb = nyo0 + (float)(2 * q + 1);
            VY[q] = make_float2(__fmaf_rn(na, F.dv_h, __fmul_rn(na, F.dv_l)), __fmaf_rn(nb, F.dv_h, __fmul_rn(nb, F.dv_l)));
            VYN[q] = make_float2(-VY[q].x, -VY[q].y);
            SR[q] = SI[q] = make_float2(0.f, 0.f);
        }
        const float2 VX = make_float2(vx, vx);
        if (P > 1) {
            const float tr = S.coef[4 + 2 * (P - 2)], ti = S.coef[5 + 2 * (P - 2)];
#pragma unroll
            for (int q = 0; q < H; ++q) {
                SR[q] = make_float2(tr, tr);
                SI[q] = make_float2(ti, ti);
            }
            for (int l = P - 2; l >= 1; --l) {                // s <- s v + c'_l
                const float cr = S.coef[4 + 2 * (l - 1)], ci = S.coef[5 + 2 * (l - 1)];
                const float2 CR = make_float2(cr, cr), CI = make_float2(ci, ci);
#pragma unroll
                for (int q = 0; q < H; ++q) {
                    const float2 nr = __ffma2_rn(SI[q], VYN[q], __ffma2_rn(SR[q], VX, CR));
                    const float2 ni = __ffma2_rn(SR[q], VY[q], __ffma2_rn(SI[q], VX, CI));
                    SR[q] = nr;
                    SI[q] = ni;
                }
            }
#pragma unroll
            for (int q = 0; q < H; ++q) {                     // s <- s v
                const float2 nr = __ffma2_rn(SI[q], VYN[q], __fmul2_rn(SR[q], VX));
                const float2 ni = __ffma2_rn(SR[q], VY[q], __fmul2_rn(SI[q], VX));
                SR[q] = nr;
                SI[q] = ni;
            }
        }
        // float-float sums of S = -alpha without c'_0 (folded into the pixel bases below):
        // the series remainder contributes -conj(s) = (-Re s, +Im s)
#pragma unroll
        for (int q = 0; q < H; ++q) {
            SXh[q] = make_float2(-SR[q].x, -SR[q].y);
            SYh[q] = SI[q];
            SXl[q] = SYl[q] = make_float2(0.f, 0.f);
        }
    }

    // ---- the block's near lenses, exactly, relative to the tile centre ----
    const unsigned long long off0 = F.near_off[blk];
    const long long n_near = (long long)(F.near_off[blk + 1] - off0);
    unsigned onlens = 0;
    if (n_near > 0) {
        const float dlt = M.delta_f, dll = M.delta_l;
        // tile centre offset from the block centre (float-float): k lattice steps, k integer
        const float kx = (float)(int)(ib - ibB + 32 - bw / 2), ky = (float)(int)(jb - jbB + 16 - bh / 2);
        const float txh = __fmul_rn(kx, dlt), txl = __fmaf_rn(kx, dll, __fmaf_rn(kx, dlt, -txh));
        const float tyh = __fmul_rn(ky, dlt), tyl = __fmaf_rn(ky, dll, __fmaf_rn(ky, dlt, -tyh));
        const float rxn = (float)iloc - 31.5f;
        const float rx = __fmaf_rn(rxn, dlt, __fmul_rn(rxn, dll));
        // per row pair q (rows 2q, 2q + 1): -y offsets of the rays, and the FP32 partial sums; the
        // near terms of a row pair go through packed f32x2 operations (each lane rounds as the
        // scalar operation would)
        float2 RYN[H], NXS[H], NYS[H];
#pragma unroll
        for (int q = 0; q < H; ++q) {
            const float na = (float)(jloc0 + 2 * q) - 15.5f, nb = (float)(jloc0 + 2 * q + 1) - 15.5f;
            RYN[q] = make_float2(-__fmaf_rn(na, dlt, __fmul_rn(na, dll)), -__fmaf_rn(nb, dlt, __fmul_rn(nb, dll)));
            NXS[q] = NYS[q] = make_float2(0.f, 0.f);
        }
        const float hx = 32.0f * dlt + kNearRadius, hy = 16.0f * dlt + kNearRadius;
        for (long long c0 = 0; c0 < n_near; c0 += kNearCap) {
            if (S.chunk0 != c0) {                             // long near list: stage this chunk
                __syncthreads();
                far_stage(M, F, blk, c0, false, S);
                __syncthreads();
            }
            const int cnt = (int)min((long long)kNearCap, n_near - c0);
            for (int j0 = 0; j0 < cnt; j0 += kNearFold) {
                for (int j = j0; j < min(cnt, j0 + kNearFold); ++j) {
                    const float4 L = S.nl[j];
                    const float lx = __fadd_rn(__fsub_rn(L.x, txh), __fsub_rn(L.y, txl));   // from the tile centre
                    const float ly = __fadd_rn(__fsub_rn(L.z, tyh), __fsub_rn(L.w, tyl));
                    if (fabsf(lx) < hx && fabsf(ly) < hy) {   // within kNearRadius of the tile: FP64
                        const int g = S.ng[j];
                        const double xl = M.lx[g], yl = M.ly[g];
                        const double ml = MASS ? M.lm[g] : 1.0;
                        const double x1 = ((double)(ib + iloc) + 0.5 - M.half_nx) * M.delta;
#pragma unroll
                        for (int r = 0; r < K; ++r) {
                            const double x2 = ((double)(jb + jloc0 + r) + 0.5 - M.half_ny) * M.delta;
                            const double d1 = xl - x1, d2 = yl - x2;
                            const double r2 = d1 * d1 + d2 * d2;
                            if (r2 == 0.0) {
                                onlens |= 1u << r;
                            } else {
                                const double t = ml / r2;
                                add_ff(lane(SXh[r >> 1], r & 1), lane(SXl[r >> 1], r & 1), t * d1);
                                add_ff(lane(SYh[r >> 1], r & 1), lane(SYl[r >> 1], r & 1), t * d2);
                            }
                        }
                        continue;
                    }
                    const float dX = __fsub_rn(lx, rx);
                    const float2 DX = make_float2(dX, dX), DX2 = dup2(__fmul_rn(dX, dX)), LY = make_float2(ly, ly);
                    const float2 MM = dup2(MASS ? S.nm[j] : 1.f);
#pragma unroll
                    for (int q = 0; q < H; ++q) {
                        const float2 dY = __fadd2_rn(LY, RYN[q]);                 // ly - ry
                        const float2 r2 = __ffma2_rn(dY, dY, DX2);
                        float2 t = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
                        if (MASS) t = __fmul2_rn(MM, t);
                        NXS[q] = __ffma2_rn(t, DX, NXS[q]);
                        NYS[q] = __ffma2_rn(t, dY, NYS[q]);
                    }
                }
#pragma unroll
                for (int r = 0; r < K; ++r) {                 // compensated fold every kNearFold lenses
                    float s, e;
                    float &xh = lane(SXh[r >> 1], r & 1), &xl = lane(SXl[r >> 1], r & 1);
                    float &yh = lane(SYh[r >> 1], r & 1), &yl = lane(SYl[r >> 1], r & 1);
                    two_sum(xh, lane(NXS[r >> 1], r & 1), s, e);
                    xh = s;
                    xl = __fadd_rn(xl, e);
                    two_sum(yh, lane(NYS[r >> 1], r & 1), s, e);
                    yh = s;
                    yl = __fadd_rn(yl, e);
                }
#pragma unroll
                for (int q = 0; q < H; ++q) NXS[q] = NYS[q] = make_float2(0.f, 0.f);
            }
        }
    }

    // ---- lens equation and pixel (float-float), as in the exact FP32 kernel ----
    const float kxh = B.kxh, kxl = B.kxl, kyh = B.kyh, kyl = B.kyl;
    // the descriptor's fields in registers for the rows below (atomics may alias it)
    const unsigned nside = (unsigned)M.nside, npix = nside * nside;
    unsigned *const counts = M.counts;
    const int rows_valid = (int)min((long long)K, max(0LL, M.j0 + M.nj - (jb + jloc0)));   // rows r < this are in the grid
    const float nsf = (float)nside;
    const long long gi = ib + iloc;
    float uxh, uxl;
    ff_axis(M.ax_h, M.ax_l, (float)(int)(2 * gi + 1 - M.nx), kxh, uxh, uxl);
    uxl = __fadd_rn(uxl, kxl);
    const bool col_ok = gi < M.i0 + M.ni;
    if (!DUMP) cnt_out += col_ok ? (unsigned)rows_valid : 0u;    // valid rays; out = valid - in (per warp)
    const float ay0 = (float)(int)(2 * (jb + jloc0) + 1 - M.ny);     // |2 j + 1 - ny| < 2^23: exact steps
    const float2 m1 = dup2(-1.f), iph = dup2(M.ip_h), niph = dup2(-M.ip_h), ipl = dup2(M.ip_l);
    const float2 ayh = dup2(M.ay_h), nayh = dup2(-M.ay_h), ayl = dup2(M.ay_l);
    const float2 UXH = dup2(uxh), UXL = dup2(uxl);
#pragma unroll
    for (int q = 0; q < H; ++q) {
        float2 uyh, uyl;
        ff_axis2(ayh, nayh, ayl, make_float2(ay0 + (float)(4 * q), ay0 + (float)(4 * q + 2)), dup2(kyh), m1, uyh, uyl);
        uyl = __fadd2_rn(uyl, dup2(kyl));
        const float2 I1 = ff_pixel2(UXH, UXL, SXh[q], SXl[q], iph, niph, ipl, m1);
        const float2 I2 = ff_pixel2(uyh, uyl, SYh[q], SYl[q], iph, niph, ipl, m1);
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int r = 2 * q + l;
            const float i1 = l ? I1.y : I1.x, i2 = l ? I2.y : I2.x;
            const bool valid = col_ok && r < rows_valid;
            const bool inside =
                valid && !((onlens >> r) & 1u) && i1 >= 0.f && i1 < nsf && i2 >= 0.f && i2 < nsf;
            const unsigned pix = inside ? (unsigned)i2 * nside + (unsigned)i1 : 0xffffffffu;
            if (DUMP) {                                       // alpha = conj(c'_0) - S
                const float xh = l ? SXh[q].y : SXh[q].x, xl = l ? SXl[q].y : SXl[q].x;
                const float yh = l ? SYh[q].y : SYh[q].x, yl = l ? SYl[q].y : SYl[q].x;
                emit_ray<true>(A, M, item, iloc + kTileX * (jloc0 + r), valid, inside, pix,
                               ((double)S.coef[0] + (double)S.coef[1]) - ((double)xh + (double)xl),
                               -((double)S.coef[2] + (double)S.coef[3]) - ((double)yh + (double)yl), cnt_in, cnt_out);
            } else {
                far_bin(counts, npix, A.check, inside, pix, cnt_in);
            }
        }
    }
}

// Production: persistent over work items of all maps of the launch. An item is a
// group of F.rows_per_item tile rows of one block (all its tile columns); its series
// and near lenses are staged once, and the next item is fetched ahead.
template <bool MASS>
__device__ void far_item(const LaunchArgs &A, const FarDesc &F, const MapDesc &M, unsigned long long it, SmemFar &S,
                         unsigned &ci, unsigned &co)
{
    const long long gpb = F.bt / F.rows_per_item;             // items per block
    const long long blk = (long long)(it / (unsigned long long)gpb);
    const long long grp = (long long)(it % (unsigned long long)gpb);
    if (!MM_BOUNDS(A.check, blk < F.nblocks, kChkFarBlock)) return;
    far_stage(M, F, blk, 0, true, S);
    __syncthreads();
    const long long bx = blk % F.blocks_x, by = blk / F.blocks_x;
    const FarBase B = far_base(M, S);
    const long long tiles_y = (M.nj + kTileY - 1) / kTileY;
    for (long long ty = by * F.bt + grp * F.rows_per_item; ty < by * F.bt + (grp + 1) * F.rows_per_item; ++ty) {
        if (ty >= tiles_y) break;
        for (long long tx = bx * F.bt; tx < (bx + 1) * F.bt && tx < M.tiles_x; ++tx)
            far_tile<false, MASS>(A, F, M, blk, bx, by, B, tx, ty, 0, S, ci, co);
    }
}

__global__ void __launch_bounds__(kShootThreads, 2) k_shoot_far(const LaunchArgs A, const FarDesc *far,
                                                             unsigned long long total_items)
{
    __shared__ SmemFar S;
    const int tid = threadIdx.x;
    const int n_maps = A.hdr->n_maps;
    if (tid == 0) S.next = atomicAdd(A.work_counter, 1ULL);
    __syncthreads();
    for (;;) {
        const unsigned long long g = S.next;
        if (g >= total_items) break;
        if (tid == 0) {
            S.red_in = 0;
            S.red_out = 0;
        }
        __syncthreads();                                      // every thread has read S.next
        if (tid == 0) S.next = atomicAdd(A.work_counter, 1ULL);
        int lo = 0, hi = n_maps - 1;                          // last map with item_begin <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (far[mid].item_begin <= g) lo = mid; else hi = mid - 1;
        }
        const MapDesc &M = A.maps[lo];
        const FarDesc &F = far[lo];
        unsigned ci = 0, co = 0;
        const unsigned long long it = F.item_first + (g - F.item_begin);
        if (M.unit_mass) far_item<false>(A, F, M, it, S, ci, co);
        else far_item<true>(A, F, M, it, S, ci, co);
        ci = __reduce_add_sync(kFull, ci);
        co = __reduce_add_sync(kFull, co) - ci;               // valid rays of the warp minus those in the map
        if ((tid & 31) == 0) {
            atomicAdd(&S.red_in, ci);
            atomicAdd(&S.red_out, co);
        }
        __syncthreads();                                      // also: shared data of this item consumed
        if (tid == 0) {
            if (S.red_in) atomicAdd(M.totals + 0, (unsigned long long)S.red_in);
            if (S.red_out) atomicAdd(M.totals + 1, (unsigned long long)S.red_out);
        }
    }
}

// Debug dump: the tiles of the request through the same tile code, one tile per item.
__global__ void __launch_bounds__(kShootThreads, 2) k_shoot_far_dump(const LaunchArgs A, const FarDesc *far)
{
    __shared__ SmemFar S;
    persistent_loop<true>(A, S.loop, [&](const MapDesc &M, unsigned long long tile, int, int item, unsigned &ci,
                                         unsigned &co) {
        const FarDesc &F = far[&M - A.maps];
        const long long tx = (long long)(tile % (unsigned long long)M.tiles_x);
        const long long ty = (long long)(tile / (unsigned long long)M.tiles_x);
        const long long blk = (ty / F.bt) * F.blocks_x + tx / F.bt;
        if (!MM_BOUNDS(A.check, blk < F.nblocks, kChkFarBlock)) return;
        __syncthreads();
        far_stage(M, F, blk, 0, true, S);
        __syncthreads();
        const FarBase B = far_base(M, S);
        if (M.unit_mass) far_tile<true, false>(A, F, M, blk, tx / F.bt, ty / F.bt, B, tx, ty, item, S, ci, co);
        else far_tile<true, true>(A, F, M, blk, tx / F.bt, ty / F.bt, B, tx, ty, item, S, ci, co);
    });
}

// ---- grouped far lenses: block setup by a walk of the lens tree ----------------
//
// One warp per block (4 per CTA). The warp walks the lens tree from the root, up to 32
// nodes per step (lane l takes the l-th newest entry of its stack), in a fixed order:
//   * a cell with |D| - r_C >= rho / q and rho + r_C <= theta |D| (D = z_C - z_B, FP64
//     with explicit roundings, as the oracle decides) is grouped: its K moments enter the
//     lane's series, c_l += -sum_k (-1)^k C(l+k, k) a_k / D^(l+k+1), and its remainder
//     (M_C / |D|) E(rho / |D|, r_C / |D|) the lane's bound;
//   * a leaf that is not grouped gives its lenses to the whole warp (lanes over lenses):
//     a lens is near by the FP32 test of the ungrouped setup; a far lens adds its FP64 series
//     terms -m / d^(l+1) and its tail m t^P / (|d| (1 - t)) to the lane's sums;
//   * any other node pushes its children.
// The lanes' sums are reduced in a fixed butterfly at the end. The count pass writes the
// near counts, the coefficients (c'_l = rho^l c_l; c'_0 as float-float) and the bound; the
// fill pass repeats the walk and writes the near lists.
constexpr int kGroupThreads = 128;

struct Cx {
    double r, i;
};

__device__ __forceinline__ Cx cmul(Cx a, Cx b)
{
    return {__dsub_rn(__dmul_rn(a.r, b.r), __dmul_rn(a.i, b.i)), __dadd_rn(__dmul_rn(a.r, b.i), __dmul_rn(a.i, b.r))};
}

__device__ __forceinline__ Cx cinv(Cx a)
{
    const double d = __dadd_rn(__dmul_rn(a.r, a.r), __dmul_rn(a.i, a.i));
    return {__ddiv_rn(a.r, d), __ddiv_rn(-a.i, d)};
}

// sum_{k>=K} C(l+k, k) y^k (the oracle's rule): the first four terms exactly, the rest bounded by a
// geometric series of the last ratio y (l+k+1)/(k+1), which falls with k; yK = y^K.
__device__ double group_tail(int l, int K, double y, double yK, const double *binom)
{
    double term = binom[(l + K) * kBinomN + K] * yK;
    double sum = 0.0;
    for (int k = K; k < K + 100000; ++k) {
        sum += term;
        const double r = y * (double)(l + k + 1) / (double)(k + 1);
        term *= r;
        if (k >= K + 3 && r < 1.0) return sum + term / (1.0 - r);
    }
    return __longlong_as_double(0x7ff0000000000000LL);       // +inf: no bound
}

template <int PMAX>
__global__ void __launch_bounds__(kGroupThreads) k_far_group(const MapDesc M, const FarDesc F, float *coef,
                                                             unsigned long long *cnt, int *near_idx)
{
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * kGroupThreads + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * kGroupThreads) >> 5;
    int *const stack = F.stack + gw * kGroupStack;
    const TreeView &T = F.tree;
    const int P = F.order, K = F.group;
    const bool fill = near_idx != nullptr;
    for (long long b = gw; b < F.nblocks; b += nw) {
        double xb, yb;
        far_centre(M, F, b % F.blocks_x, b / F.blocks_x, xb, yb);
        float cxh, cxl, cyh, cyl;
        split_d(xb, cxh, cxl);
        split_d(yb, cyh, cyl);
        double cr[PMAX], ci[PMAX];
#pragma unroll
        for (int l = 0; l < PMAX; ++l) cr[l] = ci[l] = 0.0;
        double bnd = 0.0;
        unsigned long long nnear = 0, out = fill ? F.near_off[b] : 0ULL;
        if (lane == 0) stack[0] = 0;
        int sp = 1;
        bool ovf = false;
        __syncwarp();
        while (sp > 0 && !ovf) {
            const int take = min(sp, 32);
            const int v = lane < take ? stack[sp - take + lane] : -1;
            sp -= take;
            __syncwarp();                                   // the stack entries are read before new pushes
            bool leaf = false;
            int nch = 0;
            if (v >= 0) {
                const double2 zc = T.centre[v];
                const double dx = __dsub_rn(zc.x, xb), dy = __dsub_rn(zc.y, yb);
                const double dabs = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
                const double rc = T.rc[v];
                const bool grouped = __dsub_rn(dabs, rc) >= F.rn64 && __dadd_rn(F.rho64, rc) <= __dmul_rn(F.theta, dabs);
                if (grouped) {
                    if (!fill) {
                        const Cx u = cinv({dx, dy});
                        Cx up = u;                          // u^(k+1)
                        double sr[PMAX], si[PMAX];
#pragma unroll
                        for (int l = 0; l < PMAX; ++l) sr[l] = si[l] = 0.0;
                        for (int k = 0; k < K; ++k) {
                            const double2 a = T.mom[(long long)v * K + k];
                            const Cx t = cmul({a.x, a.y}, up);
                            const double sg = (k & 1) ? 1.0 : -1.0;          // -(-1)^k
#pragma unroll
                            for (int l = 0; l < PMAX; ++l) {
                                if (l < P) {
                                    const double c = sg * T.binom[(l + k) * kBinomN + k];
                                    sr[l] = fma(c, t.r, sr[l]);
                                    si[l] = fma(c, t.i, si[l]);
                                }
                            }
                            up = cmul(up, u);
                        }
                        Cx pw = {1.0, 0.0};                 // u^l
#pragma unroll
                        for (int l = 0; l < PMAX; ++l) {
                            if (l < P) {
                                const Cx q = cmul({sr[l], si[l]}, pw);
                                cr[l] += q.r;
                                ci[l] += q.i;
                                pw = cmul(pw, u);
                            }
                        }
                        const double x = F.rho64 / dabs, y = rc / dabs, yK = pow(y, (double)K);
                        double e = pow(x / (1.0 - y), (double)P) / (1.0 - x - y), xl = 1.0;
                        for (int l = 0; l < P; ++l) {
                            e += xl * group_tail(l, K, y, yK, T.binom);
                            xl *= x;
                        }
                        bnd += T.mass[v] / dabs * e;
                    }
                } else if (T.nchild[v] == 0) {
                    leaf = true;
                } else {
                    nch = T.nchild[v];
                }
            }
            // children onto the stack, in lane order
            int pre = nch;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, pre, o);
                if (lane >= o) pre += y;
            }
            const int total = __shfl_sync(kFull, pre, 31);
            pre -= nch;
            if (sp + total > kGroupStack) {
                ovf = true;                                 // warp-uniform
            } else {
                for (int c = 0; c < nch; ++c) stack[sp + pre + c] = T.first_child[v] + c;
                sp += total;
            }
            __syncwarp();
            // the leaves of this step, in lane order, their lenses over the lanes
            unsigned lm = __ballot_sync(kFull, leaf);
            while (lm && !ovf) {
                const int src = __ffs(lm) - 1;
                lm &= lm - 1u;
                const int lv = __shfl_sync(kFull, v, src);
                const int lb = T.begin[lv], le = T.end[lv];
                for (int e0 = lb; e0 < le; e0 += 32) {
                    const int e = e0 + lane;
                    bool nr = false, fr = false;
                    int g = 0;
                    if (e < le) {
                        g = T.perm[e];
                        float ddx, ddy, r2;
                        far_offset(M.lh[g], cxh, cxl, cyh, cyl, ddx, ddy, r2);
                        nr = r2 < F.rn2;
                        fr = !nr;
                    }
                    const unsigned nb = __ballot_sync(kFull, nr);
                    if (fill) {
                        const unsigned long long at = out + __popc(nb & ((1u << lane) - 1u));
                        if (nr && MM_BOUNDS(F.check, at < F.near_off[b + 1], kChkNearList)) near_idx[at] = g;
                        out += __popc(nb);
                    } else {
                        nnear += __popc(nb);
                        if (fr) {
                            const Cx d = {__dsub_rn(M.lx[g], xb), __dsub_rn(M.ly[g], yb)};
                            const Cx u = cinv(d);
                            const double m = M.unit_mass ? 1.0 : M.lm[g];
                            Cx t = {-m * u.r, -m * u.i};
#pragma unroll
                            for (int l = 0; l < PMAX; ++l) {
                                if (l < P) {
                                    cr[l] += t.r;
                                    ci[l] += t.i;
                                    t = cmul(t, u);
                                }
                            }
                            const double da = __dsqrt_rn(__dadd_rn(__dmul_rn(d.r, d.r), __dmul_rn(d.i, d.i)));
                            const double tt = F.rho64 / da;
                            bnd += m * pow(tt, (double)P) / (da * (1.0 - tt));
                        }
                    }
                }
            }
        }
        if (ovf) {
            if (lane == 0) atomicExch(F.overflow, 1u);
            continue;
        }
        if (fill) continue;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int l = 0; l < PMAX; ++l) {
                if (l < P) {
                    cr[l] += __shfl_xor_sync(kFull, cr[l], o);
                    ci[l] += __shfl_xor_sync(kFull, ci[l], o);
                }
            }
            bnd += __shfl_xor_sync(kFull, bnd, o);
        }
        if (lane == 0) {
            cnt[b] = nnear;
            float *cb = coef + b * (long long)F.stride;
            float h, l0;
            split_d(cr[0], h, l0);
            cb[0] = h;
            cb[1] = l0;
            split_d(ci[0], h, l0);
            cb[2] = h;
            cb[3] = l0;
            double rl = 1.0;
#pragma unroll
            for (int l = 1; l < PMAX; ++l) {
                if (l < P) {
                    rl *= F.rho64;
                    cb[4 + 2 * (l - 1)] = __double2float_rn(cr[l] * rl);
                    cb[5 + 2 * (l - 1)] = __double2float_rn(ci[l] * rl);
                }
            }
            atomicMax(F.bound_max, __float_as_uint(__double2float_ru(bnd)));
        }
    }
}

}  // namespace
}  // namespace dev

int far_group_warps(int sms) { return sms * 4 * (dev::kGroupThreads / 32); }

cudaError_t launch_far_group(const MapDesc &M, const FarDesc &F, float *coef, unsigned long long *a, int *near_idx,
                             int warps, cudaStream_t s)
{
    const int grid = std::max(1, warps / (dev::kGroupThreads / 32));
    if (F.order <= 8) dev::k_far_group<8><<<grid, dev::kGroupThreads, 0, s>>>(M, F, coef, a, near_idx);
    else dev::k_far_group<16><<<grid, dev::kGroupThreads, 0, s>>>(M, F, coef, a, near_idx);
    return cudaGetLastError();
}

cudaError_t launch_far_count(const MapDesc &M, const FarDesc &F, unsigned long long *a, int grid, cudaStream_t s)
{
    dev::k_far_count<<<grid, kFarThreads, 0, s>>>(M, F, a);
    return cudaGetLastError();
}

cudaError_t launch_far_scan(unsigned long long *a, long long n, cudaStream_t s)
{
    dev::k_far_scan<<<1, 1024, 0, s>>>(a, n);
    return cudaGetLastError();
}

cudaError_t launch_far_setup(const MapDesc &M, const FarDesc &F, float *coef, int *near_idx, int grid,
                             cudaStream_t s)
{
    dev::k_far_fill<<<grid, kFarThreads, 0, s>>>(M, F, near_idx);
    const bool mass = !M.unit_mass;
    if (F.order <= 8) {
        if (mass) dev::k_far_setup<8, true><<<grid, kFarThreads, 0, s>>>(M, F, coef);
        else dev::k_far_setup<8, false><<<grid, kFarThreads, 0, s>>>(M, F, coef);
    } else if (F.order <= 16) {
        if (mass) dev::k_far_setup<16, true><<<grid, kFarThreads, 0, s>>>(M, F, coef);
        else dev::k_far_setup<16, false><<<grid, kFarThreads, 0, s>>>(M, F, coef);
    } else {
        if (mass) dev::k_far_setup<32, true><<<grid, kFarThreads, 0, s>>>(M, F, coef);
        else dev::k_far_setup<32, false><<<grid, kFarThreads, 0, s>>>(M, F, coef);
    }
    return cudaGetLastError();
}

cudaError_t launch_shoot_far(const LaunchArgs &args, const FarDesc *far, unsigned long long total_items, int grid,
                             bool dump, cudaStream_t s)
{
    if (dump) dev::k_shoot_far_dump<<<grid, dev::kShootThreads, 0, s>>>(args, far);
    else dev::k_shoot_far<<<grid, dev::kShootThreads, 0, s>>>(args, far, total_items);
    return cudaGetLastError();
}

int far_ctas_per_sm() { return 2; }

// ---- host: per-map preparation ------------------------------------------------

void far_release(MapObj &m)
{
    if (!m.arena) return;
    m.arena->free(m.far_coef);
    m.arena->free(m.far_off);
    m.arena->free(m.far_idx);
    m.arena->free(m.far_bmax);
    m.far_coef = nullptr;
    m.far_off = nullptr;
    m.far_idx = nullptr;
    m.far_bmax = nullptr;
}

// Costs of the block-size model, fitted to GB300 timings of the Fig. 1 map (558 lenses,
// 1.3e10 rays) and the sigma = 0.8 map (25 000 lenses, 9.4e10 rays) at blocks of 8 and
// 16 tiles: block preparation per block, lens and series term; near-lens work per ray and
// near lens; and a small cost per block (launch work, coefficients), which also breaks ties.
constexpr double kSetupCost = 2.15e-12;      // seconds per block x lens x term
constexpr double kNearCost = 0.81e-12;       // seconds per ray x near lens
constexpr double kBlockCost = 2.0e-9;        // seconds per block

// Grouped setup: the lens-tree walk of a block prices its grouped cells (about kGroupCells per
// tree level, each P (2K + 24) FP64 operations with its bound) at kGroupCellCost and the lenses it
// takes one by one (those of leaves within (rho + r_leaf) / theta + r_leaf of the block, 8 P
// operations each) at kGroupLensCost seconds per operation: the walk's rates over the whole GPU,
// fitted to GB300 timings of the Fig. 1 geometry with 1e5 to 1e8 lenses at blocks of 8 to 32 tiles
// (about 1.5 to 3 us of GPU time per block), with grouping found slower at 1e5 lenses and faster
// from 3e5 on.
constexpr double kGroupCells = 50.0;
constexpr double kGroupCellCost = 1.4e-11;
constexpr double kGroupLensCost = 8.2e-13;
constexpr int kAutoGroupOrder = 24;          // K of the automatic choice (bound well below 1e-8 R_E)

// Modelled time of a map's far field with block side bt and multipole order K (0: no grouping).
static double far_cost(const Geo &g, const mm_params &p, long long nstar, double radius, int bt, int K)
{
    const double rays = (double)g.nx * (double)g.ny;
    const double density = radius > 0.0 ? (double)nstar / (M_PI * radius * radius) : 0.0;
    const double bw = 64.0 * bt, bh = 32.0 * bt;
    const double blocks = std::ceil((double)g.nx / bw) * std::ceil((double)g.ny / bh);
    const double rho = g.delta * std::sqrt(0.25 * (bw * bw + bh * bh));
    const double near = density * M_PI * (rho / p.far_ratio) * (rho / p.far_ratio);
    double setup = blocks * (double)nstar * (double)p.far_order * kSetupCost;
    if (K > 0) {
        const double levels = std::max(1.0, std::log((double)std::max(nstar, 1LL) / p.far_group_leaf) / std::log(4.0));
        const double r_leaf = density > 0.0 ? std::sqrt(p.far_group_leaf / density) * 0.7071 : 0.0;
        const double reach = (rho + r_leaf) / p.far_group_theta + r_leaf;
        const double alone = std::min((double)nstar, density * M_PI * reach * reach);
        setup = blocks * (kGroupCells * levels * p.far_order * (2.0 * K + 24.0) * kGroupCellCost +
                          alone * 8.0 * p.far_order * kGroupLensCost);
    }
    return setup + rays * near * kNearCost + blocks * kBlockCost;
}

// The far field's plan for a map: block side (p.far_block, or the modelled best) and multipole
// order (p.far_group_order, or for -1 grouping with K = 24 when the model finds it faster).
// Computed from the whole ray grid, so that every part of a map (mm_shoot_into) plans alike.
static void far_plan(const Geo &g, const mm_params &p, long long nstar, double radius, int *bt_out, int *k_out)
{
    const bool can_group = nstar > 0 && p.far_order <= kGroupMaxSeries;
    int ks[2] = {0, kAutoGroupOrder}, nk = 2;
    if (p.far_group_order >= 0) {
        ks[0] = p.far_group_order;
        nk = 1;
    } else if (!can_group) {
        nk = 1;
    }
    double best = 0.0;
    int best_bt = 8, best_k = ks[0];
    for (int q = 0; q < nk; ++q) {
        for (int bt = 1; bt <= kFarMaxBlock; bt *= 2) {
            if (p.far_block > 0 && bt != 1) break;
            const int side = p.far_block > 0 ? p.far_block : bt;
            const double c = far_cost(g, p, nstar, radius, side, ks[q]);
            if ((q == 0 && bt == 1) || c < best) {
                best = c;
                best_bt = side;
                best_k = ks[q];
            }
        }
    }
    *bt_out = best_bt;
    *k_out = best_k;
}

int far_group_for(const Geo &g, const mm_params &p, long long nstar, double radius)
{
    int bt, K;
    far_plan(g, p, nstar, radius, &bt, &K);
    return K;
}

int far_block_for(const Geo &g, const mm_params &p, long long nstar, double radius)
{
    int bt, K;
    far_plan(g, p, nstar, radius, &bt, &K);
    return bt;
}

int far_prepare(mm_ctx *ctx, MapObj &m, cudaStream_t s, unsigned int *check)
{
    far_release(m);
    const Geo &g = m.g;
    const mm_params &p = m.p;
    FarDesc &F = m.far;
    F = FarDesc{};
    F.order = p.far_order;
    F.bt = far_block_for(g, p, m.lenses->n, m.lenses->radius);
    const long long bw = 64LL * F.bt, bh = 32LL * F.bt;
    F.blocks_x = (g.ni + bw - 1) / bw;
    F.blocks_y = (g.nj + bh - 1) / bh;
    F.nblocks = F.blocks_x * F.blocks_y;
    F.stride = (4 + 2 * (F.order - 1) + 3) & ~3;
    // whole blocks as work items when there are enough of them to fill the GPU, else tile rows
    const long long ctas = (long long)ctx->sms * far_ctas_per_sm();
    F.rows_per_item = F.nblocks >= 4 * ctas ? F.bt : 1;
    F.items = (unsigned long long)F.nblocks * (unsigned long long)(F.bt / F.rows_per_item);
    F.item_begin = 0;
    const double rho = g.delta * std::sqrt((double)(bw / 2) * (double)(bw / 2) + (double)(bh / 2) * (double)(bh / 2));
    const double rn = rho / p.far_ratio;
    F.rn2 = (float)(rn * rn);
    F.rho = (float)rho;
    const double dv = g.delta / rho;
    F.dv_h = (float)dv;
    F.dv_l = (float)(dv - (double)F.dv_h);
    int rc;
    if ((rc = ctx->arena.alloc(sizeof(unsigned), (void **)&m.far_bmax))) return rc;
    MM_CUDA(cudaMemsetAsync(m.far_bmax, 0, sizeof(unsigned), s));
    F.bound_max = m.far_bmax;
    F.check = check;                                // the caller's bounds-check word
    if (F.nblocks == 0) return MM_OK;
    if ((rc = ctx->arena.alloc((size_t)F.nblocks * F.stride * sizeof(float), (void **)&m.far_coef)) ||
        (rc = ctx->arena.alloc((size_t)(F.nblocks + 1) * sizeof(unsigned long long), (void **)&m.far_off)))
        return rc;
    MapDesc d;
    fill_desc(m, &d);
    const int K = far_group_for(g, p, m.lenses->n, m.lenses->radius);
    if (K > 0 && m.lenses->n > 0) {              // grouped far lenses: walk the lens set's tree
        {
            std::lock_guard<std::mutex> lk(m.lenses->tree_mu);
            if ((rc = build_lens_tree(ctx, *m.lenses, K, p.far_group_leaf, s))) return rc;
            F.tree = m.lenses->tree.view();
        }
        F.group = K;
        F.theta = p.far_group_theta;
        F.rho64 = rho;
        F.rn64 = rn;
        F.coef = m.far_coef;
        F.near_off = m.far_off;
        const int warps = far_group_warps(ctx->sms);
        struct Tmp {
            DeviceArena *a;
            std::vector<void *> v;
            ~Tmp() { for (void *q : v) a->free(q); }
        } tmp{&ctx->arena, {}};
        if ((rc = ctx->arena.alloc((size_t)warps * kGroupStack * sizeof(int), (void **)&F.stack))) return rc;
        tmp.v.push_back(F.stack);
        if ((rc = ctx->arena.alloc(sizeof(unsigned), (void **)&F.overflow))) return rc;
        tmp.v.push_back(F.overflow);
        MM_CUDA(cudaMemsetAsync(F.overflow, 0, sizeof(unsigned), s));
        MM_CUDA(launch_far_group(d, F, m.far_coef, m.far_off, nullptr, warps, s));
        unsigned ovf = 0;
        MM_CUDA(cudaMemcpyAsync(&ovf, F.overflow, sizeof(ovf), cudaMemcpyDeviceToHost, s));
        MM_CUDA(cudaStreamSynchronize(s));
        if (ovf) return fail(MM_EINVAL, "far field: the lens-tree walk of a block outgrew its stack (lower far_block "
                                        "or raise far_group_leaf)");
        if ((rc = scan_exclusive(ctx, m.far_off, F.nblocks, s))) return rc;
        unsigned long long total = 0;
        MM_CUDA(cudaMemcpyAsync(&total, m.far_off + F.nblocks, sizeof(total), cudaMemcpyDeviceToHost, s));
        MM_CUDA(cudaStreamSynchronize(s));
        if (total > (unsigned long long)INT32_MAX) return fail(MM_ENOMEM, "far field: near lists too long (lower far_block)");
        if ((rc = ctx->arena.alloc(std::max<size_t>(1, (size_t)total) * sizeof(int), (void **)&m.far_idx))) return rc;
        F.near_idx = m.far_idx;
        MM_CUDA(launch_far_group(d, F, m.far_coef, m.far_off, m.far_idx, warps, s));
        MM_CUDA(cudaStreamSynchronize(s));            // the stack goes back to the arena
        F.stack = nullptr;
        F.overflow = nullptr;
        return MM_OK;
    }
    const int grid = (int)std::max(1LL, std::min(F.nblocks, (long long)ctx->sms * 8));
    MM_CUDA(launch_far_count(d, F, m.far_off, grid, s));
    MM_CUDA(launch_far_scan(m.far_off, F.nblocks, s));
    unsigned long long total = 0;
    MM_CUDA(cudaMemcpyAsync(&total, m.far_off + F.nblocks, sizeof(total), cudaMemcpyDeviceToHost, s));
    MM_CUDA(cudaStreamSynchronize(s));
    if (total > (unsigned long long)INT32_MAX) return fail(MM_ENOMEM, "far field: near lists too long (lower far_block)");
    if ((rc = ctx->arena.alloc(std::max<size_t>(1, (size_t)total) * sizeof(int), (void **)&m.far_idx))) return rc;
    F.coef = m.far_coef;
    F.near_off = m.far_off;
    F.near_idx = m.far_idx;
    MM_CUDA(launch_far_setup(d, F, m.far_coef, m.far_idx, grid, s));
    return MM_OK;
}

}  // namespace mm
