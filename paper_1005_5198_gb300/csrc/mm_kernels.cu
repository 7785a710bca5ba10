// mm_kernels.cu -- sm_103a kernels for direct inverse ray-shooting.
//
// What is computed (Sect. 2, Eq. sigma, and the inverse ray-shooting
// estimator): for every ray x of the regular image-plane lattice,
//     alpha(x) = sum_i m_i (x - x_i) / |x - x_i|^2            (all N* lenses)
//     y1 = (1 - gamma - sigma_c) x1 - alpha1,  y2 = (1 + gamma - sigma_c) x2 - alpha2
// and the ray is counted into source pixel (floor((y1+L/2)/p), floor((y2+L/2)/p)).
// The smooth and shear terms are applied after the deflection sum, as the
// paper's GPU code does (Sect. 2.3, the recast lens equation).
//
// Work decomposition: a launch covers the ray tiles (64 x 32 rays) of one or
// more maps; CTAs take tiles from a device counter (persistent kernel). Each
// thread owns 8 rays of one lattice column.
//
// FP32 path (MM_FP32C):
//   * coordinates relative to the tile centre: the ray offsets are small
//     exact multiples of the spacing, the lens offsets are formed from
//     float-float lens coordinates, so far lenses lose no absolute accuracy;
//   * lens pairs (a, b) are processed with packed f32x2 FMA/ADD (one issue
//     for two lanes); the squared-distance reciprocal is either two MUFU
//     reciprocals or, for "shared-reciprocal" pairs, one reciprocal of the
//     product: 1/ra = rb / (ra rb), 1/rb = ra / (ra rb), which moves work from
//     the MUFU pipe (16/clk/SM) to the FMA pipe (128 lanes/clk/SM);
//   * lanes accumulate FP32 partial sums that are folded every FOLD pairs into
//     a float-float (hi, lo) accumulator with the error-free TwoSum
//     (Knuth; compensated summation at chunk granularity);
//   * lenses within kNearRadius of the tile's ray box are replaced by a null
//     lens in the FP32 sweep and added in FP64 instead (their terms are large
//     and would lose the absolute accuracy target in FP32);
//   * the source position and pixel come from a float-float evaluation of the
//     lens equation, accurate to ~1e-9 pixel.
// FP64 path (MM_FP64): the same tiles, every operation in FP64, summed in
// lens order -- the plain form.
#include <cuda_runtime.h>
#include <cstdint>

#include "mm_internal.h"

namespace mm {
namespace {

constexpr int K = kRaysPerThread;

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

// Add an FP64 value into a float-float accumulator.
__device__ __forceinline__ void add_ff(float &h, float &l, double v)
{
    const float vh = __double2float_rn(v);
    const float vl = __double2float_rn(v - (double)vh);
    float s, e;
    two_sum(h, vh, s, e);
    h = s;
    l = __fadd_rn(l, __fadd_rn(e, vl));
}

// Float-float u = (c_h + c_l) * n + base for an exact integer-valued float n.
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

// Pixel coordinate floor(u) with u = (uh + ul) + S/p, S = Sh + Sl (float-float).
__device__ __forceinline__ float ff_pixel(float uh, float ul, float sh, float sl, float iph, float ipl)
{
    const float th = __fmul_rn(sh, iph);
    float te = __fmaf_rn(sh, iph, -th);
    te = __fmaf_rn(sh, ipl, te);
    te = __fmaf_rn(sl, iph, te);
    float s, e;
    two_sum(uh, th, s, e);
    const float lo = __fadd_rn(__fadd_rn(e, ul), te);
    float I = floorf(s);
    const float f = __fadd_rn(__fsub_rn(s, I), lo);
    return __fadd_rn(I, floorf(f));
}

struct __align__(16) Smem {
    float4 pos[kChunkPairs];     // (xa, xb, ya, yb) relative to the tile centre
    float2 mass[kChunkPairs];    // (ma, mb)
    double2 lens64[kChunkPairs]; // FP64 path: (x, y) of lens k of the chunk (256 lenses)
    double m64[kChunkPairs];
    unsigned near_bits[2 * kThreads / 32];
    unsigned long long g;
    int map;
    int near_any;
    unsigned red_in, red_out;
    double cx, cy;               // tile centre (FP64)
};

__device__ __forceinline__ int find_map(const LaunchArgs &A, int n_maps, unsigned long long g)
{
    int lo = 0, hi = n_maps - 1;
    while (lo < hi) {                           // last map with tile_begin <= g
        const int mid = (lo + hi + 1) >> 1;
        if (A.maps[mid].tile_begin <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// First request of work item `item` whose local ray index equals `mine` (requests of
// an item are sorted by local index), or -1.
__device__ __forceinline__ int dump_find(const DumpArgs &D, int item, int mine)
{
    int lo = D.begin[item], hi = D.begin[item + 1];
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (D.local[mid] < mine) lo = mid + 1; else hi = mid;
    }
    return (lo < D.begin[item + 1] && D.local[lo] == mine) ? lo : -1;
}

// One lens pair applied to the thread's K rays.
template <bool MASS, bool SHARED_RCP>
__device__ __forceinline__ void pair_step(const float4 P, const float2 Mm, const float2 NRX,
                                          const float2 (&NRY)[K], float2 (&AX)[K], float2 (&AY)[K])
{
    const float2 LX = make_float2(P.x, P.y);
    const float2 LY = make_float2(P.z, P.w);
    const float2 dX = __fadd2_rn(LX, NRX);        // x_l - x (shared by the column's rays)
    const float2 dX2 = __fmul2_rn(dX, dX);
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const float2 dY = __fadd2_rn(LY, NRY[r]);
        const float2 R2 = __ffma2_rn(dY, dY, dX2);
        float2 W;
        if (SHARED_RCP) {
            const float q = rcp_approx(__fmul_rn(R2.x, R2.y));
            if (MASS) {
                W.x = __fmul_rn(q, __fmul_rn(R2.y, Mm.x));
                W.y = __fmul_rn(q, __fmul_rn(R2.x, Mm.y));
            } else {
                W.x = __fmul_rn(q, R2.y);
                W.y = __fmul_rn(q, R2.x);
            }
        } else {
            W.x = rcp_approx(R2.x);
            W.y = rcp_approx(R2.y);
            if (MASS) W = __fmul2_rn(W, Mm);
        }
        AX[r] = __ffma2_rn(W, dX, AX[r]);
        AY[r] = __ffma2_rn(W, dY, AY[r]);
    }
}

template <int SHARED4, int FOLD, bool MASS, bool DUMP>
__device__ void tile_fp32(const LaunchArgs &A, const MapDesc &M, unsigned long long tile, int item, Smem &S,
                          unsigned &cnt_in, unsigned &cnt_out)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int w = tid >> 5;
    const int iloc = (w & 1) * 32 + lane;
    const int jloc0 = (w >> 1) * K;
    const long long tx = (long long)(tile % (unsigned long long)M.tiles_x);
    const long long ty = (long long)(tile / (unsigned long long)M.tiles_x);
    const long long ib = M.i0 + tx * kTileX;
    const long long jb = M.j0 + ty * kTileY;
    const long long gi = ib + iloc;

    if (tid == 0) {
        S.cx = ((double)ib + 32.0 - M.half_nx) * M.delta;
        S.cy = ((double)jb + 16.0 - M.half_ny) * M.delta;
    }
    __syncthreads();
    const double cx = S.cx, cy = S.cy;
    const float cxh = __double2float_rn(cx), cxl = __double2float_rn(cx - (double)cxh);
    const float cyh = __double2float_rn(cy), cyl = __double2float_rn(cy - (double)cyh);

    const float dlt = M.delta_f;
    const float rx = __fmaf_rn((float)iloc - 31.5f, dlt, __fmul_rn((float)iloc - 31.5f, M.delta_l));
    const float2 NRX = make_float2(-rx, -rx);
    float2 NRY[K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const float ry = __fmaf_rn((float)(jloc0 + r) - 15.5f, dlt, __fmul_rn((float)(jloc0 + r) - 15.5f, M.delta_l));
        NRY[r] = make_float2(-ry, -ry);
    }
    const float hx = 32.0f * dlt + kNearRadius;
    const float hy = 16.0f * dlt + kNearRadius;

    float2 AX[K], AY[K];
    float SXh[K], SXl[K], SYh[K], SYl[K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        AX[r] = make_float2(0.f, 0.f);
        AY[r] = make_float2(0.f, 0.f);
        SXh[r] = SXl[r] = SYh[r] = SYl[r] = 0.f;
    }
    unsigned onlens = 0;

    const long long nstar = M.nstar;
    for (long long base = 0; base < nstar; base += kChunkLenses) {
        // ---- stage 256 lens pairs relative to the tile centre ----
        __syncthreads();                       // previous chunk fully consumed
        {
            const long long la = base + 2 * tid;     // lh is padded: la + 1 < padded size
            const float4 qa = M.lh[la];
            const float4 qb = M.lh[la + 1];
            float xa = __fadd_rn(__fsub_rn(qa.x, cxh), __fsub_rn(qa.z, cxl));
            float ya = __fadd_rn(__fsub_rn(qa.y, cyh), __fsub_rn(qa.w, cyl));
            float xb = __fadd_rn(__fsub_rn(qb.x, cxh), __fsub_rn(qb.z, cxl));
            float yb = __fadd_rn(__fsub_rn(qb.y, cyh), __fsub_rn(qb.w, cyl));
            const bool na = fabsf(xa) < hx && fabsf(ya) < hy;
            const bool nb = fabsf(xb) < hx && fabsf(yb) < hy;
            float ma = 1.f, mb = 1.f;
            if (MASS) { ma = M.lmf[la]; mb = M.lmf[la + 1]; }
            if (na) { xa = kNullX; ya = 0.f; ma = 0.f; }
            if (nb) { xb = kNullX; yb = 0.f; mb = 0.f; }
            S.pos[tid] = make_float4(xa, xb, ya, yb);
            if (MASS) S.mass[tid] = make_float2(ma, mb);
            const unsigned ba = __ballot_sync(0xffffffffu, na);
            const unsigned bb = __ballot_sync(0xffffffffu, nb);
            if (lane == 0) { S.near_bits[2 * w] = ba; S.near_bits[2 * w + 1] = bb; }
        }
        __syncthreads();

        // ---- FP32 sweep over the chunk's pairs ----
        long long left = nstar - base;
        int npairs = (int)((left >= kChunkLenses) ? kChunkPairs : ((left + 1) >> 1));
        npairs = (npairs + 3) & ~3;            // padded entries are null lenses
        for (int p0 = 0; p0 < npairs; p0 += FOLD) {
            const int pend = min(p0 + FOLD, npairs);
            for (int p = p0; p < pend; p += 4) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float4 P = S.pos[p + u];
                    const float2 Mm = MASS ? S.mass[p + u] : make_float2(1.f, 1.f);
                    if (u < SHARED4) pair_step<MASS, true>(P, Mm, NRX, NRY, AX, AY);
                    else pair_step<MASS, false>(P, Mm, NRX, NRY, AX, AY);
                }
            }
#pragma unroll
            for (int r = 0; r < K; ++r) {       // compensated fold of the lane partials
                float s, e;
                two_sum(SXh[r], __fadd_rn(AX[r].x, AX[r].y), s, e);
                SXh[r] = s; SXl[r] = __fadd_rn(SXl[r], e);
                two_sum(SYh[r], __fadd_rn(AY[r].x, AY[r].y), s, e);
                SYh[r] = s; SYl[r] = __fadd_rn(SYl[r], e);
                AX[r] = make_float2(0.f, 0.f);
                AY[r] = make_float2(0.f, 0.f);
            }
        }

        // ---- near lenses of this chunk, in FP64 ----
        unsigned any = 0;
#pragma unroll
        for (int k = 0; k < 2 * kThreads / 32; ++k) any |= S.near_bits[k];
        if (any) {
            const double x1 = ((double)gi + 0.5 - M.half_nx) * M.delta;
            for (int k = 0; k < 2 * kThreads / 32; ++k) {
                unsigned bits = S.near_bits[k];
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const long long g = base + 2 * (32 * (k >> 1) + b) + (k & 1);
                    const double xl = M.lx[g], yl = M.ly[g];
                    const double ml = MASS ? M.lm[g] : 1.0;
#pragma unroll
                    for (int r = 0; r < K; ++r) {
                        const double x2 = ((double)(jb + jloc0 + r) + 0.5 - M.half_ny) * M.delta;
                        const double d1 = xl - x1, d2 = yl - x2;
                        const double r2 = d1 * d1 + d2 * d2;
                        if (r2 == 0.0) {
                            onlens |= 1u << r;
                        } else {
                            const double t = ml / r2;
                            add_ff(SXh[r], SXl[r], t * d1);
                            add_ff(SYh[r], SYl[r], t * d2);
                        }
                    }
                }
            }
        }
    }

    // ---- epilogue: lens equation and pixel (float-float) ----
    float uxh, uxl;
    ff_axis(M.ax_h, M.ax_l, (float)(2 * gi + 1 - M.nx), M.half_n, uxh, uxl);
    const bool col_ok = gi < M.i0 + M.ni;
    const float nsf = (float)M.nside;
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const long long gj = jb + jloc0 + r;
        float uyh, uyl;
        ff_axis(M.ay_h, M.ay_l, (float)(2 * gj + 1 - M.ny), M.half_n, uyh, uyl);
        const float I1 = ff_pixel(uxh, uxl, SXh[r], SXl[r], M.ip_h, M.ip_l);
        const float I2 = ff_pixel(uyh, uyl, SYh[r], SYl[r], M.ip_h, M.ip_l);
        const bool valid = col_ok && gj < M.j0 + M.nj;
        const bool inside = valid && !((onlens >> r) & 1u) && I1 >= 0.f && I1 < nsf && I2 >= 0.f && I2 < nsf;
        const unsigned pix = inside ? (unsigned)I2 * (unsigned)M.nside + (unsigned)I1 : 0xffffffffu;
        if (DUMP) {
            const int mine = iloc + kTileX * (jloc0 + r);
            for (int q = dump_find(A.dump, item, mine); q >= 0 && q < A.dump.begin[item + 1] && A.dump.local[q] == mine; ++q) {
                const int sl = A.dump.slot[q];
                A.dump.alpha[2 * sl] = -((double)SXh[r] + (double)SXl[r]);
                A.dump.alpha[2 * sl + 1] = -((double)SYh[r] + (double)SYl[r]);
                A.dump.pixel[sl] = inside ? (long long)pix : -1LL;
            }
        } else {
            const unsigned peers = __match_any_sync(0xffffffffu, pix);
            if (inside && lane == __ffs(peers) - 1) atomicAdd(M.counts + pix, (unsigned)__popc(peers));
            cnt_in += inside ? 1u : 0u;
            cnt_out += (valid && !inside) ? 1u : 0u;
        }
    }
}

template <int SHARED4, int FOLD, bool DUMP>
__device__ __forceinline__ void tile_fp32_any_mass(const LaunchArgs &A, const MapDesc &M, unsigned long long tile,
                                                   int item, Smem &S, unsigned &ci, unsigned &co)
{
    if (M.unit_mass) tile_fp32<SHARED4, FOLD, false, DUMP>(A, M, tile, item, S, ci, co);
    else tile_fp32<SHARED4, FOLD, true, DUMP>(A, M, tile, item, S, ci, co);
}

template <bool DUMP>
__device__ void tile_fp32_dispatch(const LaunchArgs &A, const MapDesc &M, unsigned long long tile, int item, Smem &S,
                                   unsigned &ci, unsigned &co)
{
    switch (M.variant) {
    case 1: tile_fp32_any_mass<3, 64, DUMP>(A, M, tile, item, S, ci, co); break;
    case 2: tile_fp32_any_mass<4, 32, DUMP>(A, M, tile, item, S, ci, co); break;
    case 3: tile_fp32_any_mass<4, 64, DUMP>(A, M, tile, item, S, ci, co); break;
    case 4: tile_fp32_any_mass<2, 32, DUMP>(A, M, tile, item, S, ci, co); break;
    case 5: tile_fp32_any_mass<2, 64, DUMP>(A, M, tile, item, S, ci, co); break;
    case 6: tile_fp32_any_mass<0, 32, DUMP>(A, M, tile, item, S, ci, co); break;
    case 7: tile_fp32_any_mass<0, 64, DUMP>(A, M, tile, item, S, ci, co); break;
    default: tile_fp32_any_mass<3, 32, DUMP>(A, M, tile, item, S, ci, co); break;
    }
}

template <bool DUMP>
__device__ void tile_fp64(const LaunchArgs &A, const MapDesc &M, unsigned long long tile, int item, Smem &S,
                          unsigned &cnt_in, unsigned &cnt_out)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int w = tid >> 5;
    const int iloc = (w & 1) * 32 + lane;
    const int jloc0 = (w >> 1) * K;
    const long long tx = (long long)(tile % (unsigned long long)M.tiles_x);
    const long long ty = (long long)(tile / (unsigned long long)M.tiles_x);
    const long long ib = M.i0 + tx * kTileX;
    const long long jb = M.j0 + ty * kTileY;
    const long long gi = ib + iloc;
    const double x1 = ((double)gi + 0.5 - M.half_nx) * M.delta;
    double x2[K], a1[K], a2[K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        x2[r] = ((double)(jb + jloc0 + r) + 0.5 - M.half_ny) * M.delta;
        a1[r] = a2[r] = 0.0;
    }
    unsigned onlens = 0;
    for (long long base = 0; base < M.nstar; base += kChunkPairs) {
        __syncthreads();
        {
            const long long g = base + tid;
            if (g < M.nstar) {
                S.lens64[tid] = make_double2(M.lx[g], M.ly[g]);
                S.m64[tid] = M.lm[g];
            }
        }
        __syncthreads();
        const int n = (int)min((long long)kChunkPairs, M.nstar - base);
        for (int k = 0; k < n; ++k) {
            const double2 L = S.lens64[k];
            const double m = S.m64[k];
#pragma unroll
            for (int r = 0; r < K; ++r) {
                const double d1 = x1 - L.x, d2 = x2[r] - L.y;
                const double r2 = d1 * d1 + d2 * d2;
                if (r2 == 0.0) {
                    onlens |= 1u << r;
                } else {
                    a1[r] += m * d1 / r2;
                    a2[r] += m * d2 / r2;
                }
            }
        }
    }
    const bool col_ok = gi < M.i0 + M.ni;
    const double nsd = (double)M.nside;
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const long long gj = jb + jloc0 + r;
        const double y1 = M.one_m_gamma * x1 - M.sigma_c * x1 - a1[r];
        const double y2 = M.one_p_gamma * x2[r] - M.sigma_c * x2[r] - a2[r];
        const double u1 = floor((y1 + M.half_side) / M.pix);
        const double u2 = floor((y2 + M.half_side) / M.pix);
        const bool valid = col_ok && gj < M.j0 + M.nj;
        const bool inside = valid && !((onlens >> r) & 1u) && u1 >= 0.0 && u1 < nsd && u2 >= 0.0 && u2 < nsd;
        const unsigned pix = inside ? (unsigned)u2 * (unsigned)M.nside + (unsigned)u1 : 0xffffffffu;
        if (DUMP) {
            const int mine = iloc + kTileX * (jloc0 + r);
            for (int q = dump_find(A.dump, item, mine); q >= 0 && q < A.dump.begin[item + 1] && A.dump.local[q] == mine; ++q) {
                const int sl = A.dump.slot[q];
                A.dump.alpha[2 * sl] = a1[r];
                A.dump.alpha[2 * sl + 1] = a2[r];
                A.dump.pixel[sl] = inside ? (long long)pix : -1LL;
            }
        } else {
            const unsigned peers = __match_any_sync(0xffffffffu, pix);
            if (inside && lane == __ffs(peers) - 1) atomicAdd(M.counts + pix, (unsigned)__popc(peers));
            cnt_in += inside ? 1u : 0u;
            cnt_out += (valid && !inside) ? 1u : 0u;
        }
    }
}

// Persistent driver: take work items from the counter until exhausted; flush the
// per-map in/out ray counts whenever the map changes and at exit.
template <bool FP64, bool DUMP>
__global__ void __launch_bounds__(kThreads, FP64 ? 1 : 2) k_shoot(const LaunchArgs A)
{
    __shared__ Smem S;
    const int tid = threadIdx.x;
    int cur_map = -1;
    unsigned long long run_in = 0, run_out = 0;   // meaningful in thread 0
    const unsigned long long total_work = A.hdr->total_work;
    const int n_maps = A.hdr->n_maps;
    for (;;) {
        if (tid == 0) {
            const unsigned long long g = atomicAdd(A.work_counter, 1ULL);
            S.g = g;
            S.map = (g < total_work) ? (DUMP ? 0 : find_map(A, n_maps, g)) : -1;
            S.red_in = 0;
            S.red_out = 0;
        }
        __syncthreads();
        const unsigned long long g = S.g;
        const int mi = S.map;
        if (g >= total_work) break;
        if (tid == 0 && cur_map != mi) {
            if (cur_map >= 0 && !DUMP) {
                atomicAdd(A.maps[cur_map].totals + 0, run_in);
                atomicAdd(A.maps[cur_map].totals + 1, run_out);
            }
            cur_map = mi;
            run_in = run_out = 0;
        }
        const MapDesc &M = A.maps[mi];
        const unsigned long long tile = DUMP ? A.dump.tile[g] : M.tile_first + (g - M.tile_begin);
        const int item = DUMP ? (int)g : 0;
        unsigned ci = 0, co = 0;
        if (FP64) tile_fp64<DUMP>(A, M, tile, item, S, ci, co);
        else tile_fp32_dispatch<DUMP>(A, M, tile, item, S, ci, co);
        if (!DUMP) {
            ci = __reduce_add_sync(0xffffffffu, ci);
            co = __reduce_add_sync(0xffffffffu, co);
            if ((tid & 31) == 0) { atomicAdd(&S.red_in, ci); atomicAdd(&S.red_out, co); }
        }
        __syncthreads();
        if (tid == 0) { run_in += S.red_in; run_out += S.red_out; }
        __syncthreads();                       // S.g / S.red_* are rewritten next iteration
    }
    if (tid == 0 && cur_map >= 0 && !DUMP) {
        atomicAdd(A.maps[cur_map].totals + 0, run_in);
        atomicAdd(A.maps[cur_map].totals + 1, run_out);
    }
}

__global__ void k_prepare_lenses(const double *x, const double *y, const double *m, long long n, long long n_pad,
                                 float4 *lh, float *lmf)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n_pad;
         k += (long long)gridDim.x * blockDim.x) {
        if (k < n) {
            const double xv = x[k], yv = y[k];
            const float xh = __double2float_rn(xv), yh = __double2float_rn(yv);
            lh[k] = make_float4(xh, yh, __double2float_rn(xv - (double)xh), __double2float_rn(yv - (double)yh));
            lmf[k] = __double2float_rn(m[k]);
        } else {
            lh[k] = make_float4(kNullX, 0.f, 0.f, 0.f);
            lmf[k] = 0.f;
        }
    }
}

}  // namespace

cudaError_t launch_prepare_lenses(const double *x, const double *y, const double *m, long long n, long long n_pad,
                                  float4 *lh, float *lmf, cudaStream_t s)
{
    if (n_pad <= 0) return cudaSuccess;
    const int grid = (int)min((n_pad + 255) / 256, (long long)4096);
    k_prepare_lenses<<<grid, 256, 0, s>>>(x, y, m, n, n_pad, lh, lmf);
    return cudaGetLastError();
}

cudaError_t launch_shoot_fp32(const LaunchArgs &args, int grid, bool dump, cudaStream_t s)
{
    if (dump) k_shoot<false, true><<<grid, kThreads, 0, s>>>(args);
    else k_shoot<false, false><<<grid, kThreads, 0, s>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_shoot_fp64(const LaunchArgs &args, int grid, bool dump, cudaStream_t s)
{
    if (dump) k_shoot<true, true><<<grid, kThreads, 0, s>>>(args);
    else k_shoot<true, false><<<grid, kThreads, 0, s>>>(args);
    return cudaGetLastError();
}

int shoot_ctas_per_sm(bool fp64) { return fp64 ? 1 : 2; }

const char *variant_name(int v)
{
    static const char *names[kNumVariants] = {
        "shared-rcp 3/4, fold 32", "shared-rcp 3/4, fold 64", "shared-rcp 4/4, fold 32", "shared-rcp 4/4, fold 64",
        "shared-rcp 2/4, fold 32", "shared-rcp 2/4, fold 64", "shared-rcp 0/4, fold 32", "shared-rcp 0/4, fold 64"};
    return (v >= 0 && v < kNumVariants) ? names[v] : "invalid";
}

}  // namespace mm
