// mm_fp32.cuh -- the FP32 (compensated) shooting kernel, templated on the ray
// layout of a thread: C lattice columns x R lattice rows.
//
// What is computed (Sect. 2, Eq. sigma, and the inverse ray-shooting
// estimator): for every ray x of the regular image-plane lattice,
//     alpha(x) = sum_i m_i (x - x_i) / |x - x_i|^2            (all N* lenses)
//     y1 = (1 - gamma - sigma_c) x1 - alpha1,  y2 = (1 + gamma - sigma_c) x2 - alpha2
// and the ray is counted into source pixel (floor((y1+L/2)/p), floor((y2+L/2)/p)).
// The smooth-matter and shear terms are applied after the deflection sum, as in
// the paper's GPU code (Sect. 2.3, the recast lens equation).
//
// Work decomposition: a launch covers the 64 x 32-ray tiles of one or more maps;
// CTAs take tiles from a device counter (persistent kernel). The tile is the same
// for every layout (C, R) and every ray sees exactly the same FP32 operations in
// the same order, so all layouts give bit-identical maps; layouts differ only in
// how work is spread over threads (and so in occupancy and shared work):
//   * the x-differences to a lens pair (and their squares) are shared by a
//     thread's R rows, the y-differences by its C columns;
//   * lens pairs (a, b) are processed with packed f32x2 FMA/ADD/MUL (one issue
//     for two lanes); the squared-distance reciprocal is either two MUFU
//     reciprocals or, for "shared-reciprocal" pairs, one MUFU reciprocal of the
//     product, 1/ra = rb/(ra rb), 1/rb = ra/(ra rb), which moves work from the
//     MUFU pipe (16/clk/SM) to the FMA pipe (128 lanes/clk/SM);
//   * coordinates are relative to the tile centre: ray offsets are small
//     multiples of the spacing, lens offsets come from float-float lens
//     coordinates, so far lenses lose no absolute accuracy;
//   * lane partial sums are folded every FOLD pairs into a float-float (hi, lo)
//     accumulator with the error-free TwoSum (compensated summation);
//   * lenses within kNearRadius of the tile's ray box are replaced by a null
//     lens in the FP32 sweep and summed in FP64 instead;
//   * the source position and pixel come from a float-float evaluation of the
//     lens equation (about 1e-9 pixel).
#pragma once
#include "mm_device.cuh"

namespace mm {
namespace dev {

// Thread layout: C columns x R rows of the tile per thread; the float-float sums in
// registers (SREG) or shared memory; registers sized for MINB CTAs per SM.
template <int C, int R, bool SREG_, int MINB_>
struct Layout {
    static constexpr int NT = kTileRays / (C * R);   // threads per CTA
    static constexpr int WX = 2 / C;                  // warps along x: 64 = 32 * C * WX
    static constexpr int MINB = MINB_;
    static constexpr bool SREG = SREG_;
    static_assert(C == 1 || C == 2, "C must be 1 or 2");
    static_assert(NT % 32 == 0 && kChunkPairs % NT == 0, "layout must cover the tile and the staging chunk");
};

// Float-float sums (x_hi, x_lo, y_hi, y_lo) of a thread's rays: registers or shared memory.
template <int C, int R, bool SREG, int NT>
struct Sums;

template <int C, int R, int NT>
struct Sums<C, R, true, NT> {
    float4 v[C][R];
    __device__ __forceinline__ Sums(SmemFP32 &) {}
    __device__ __forceinline__ float4 get(int c, int r) const { return v[c][r]; }
    __device__ __forceinline__ void set(int c, int r, float4 a) { v[c][r] = a; }
};

template <int C, int R, int NT>
struct Sums<C, R, false, NT> {
    float4 *base;
    __device__ __forceinline__ Sums(SmemFP32 &S) : base(S.acc + threadIdx.x) {}
    __device__ __forceinline__ float4 get(int c, int r) const { return base[(c * R + r) * NT]; }
    __device__ __forceinline__ void set(int c, int r, float4 a) { base[(c * R + r) * NT] = a; }
};

// One lens pair applied to the thread's C x R rays.
template <int C, int R, bool MASS, bool SHARED_RCP>
__device__ __forceinline__ void pair_step(const float4 P, const float2 Mm, const float2 (&NRX)[C],
                                          const float2 (&NRY)[R], float2 (&AX)[C][R], float2 (&AY)[C][R])
{
    const float2 LX = make_float2(P.x, P.y);
    const float2 LY = make_float2(P.z, P.w);
    float2 dX[C], dX2[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        dX[c] = __fadd2_rn(LX, NRX[c]);       // x_l - x, shared by the column's R rays
        dX2[c] = __fmul2_rn(dX[c], dX[c]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float2 dY = __fadd2_rn(LY, NRY[r]);   // y_l - y, shared by the row's C rays
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float2 R2 = __ffma2_rn(dY, dY, dX2[c]);
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
            AX[c][r] = __ffma2_rn(W, dX[c], AX[c][r]);
            AY[c][r] = __ffma2_rn(W, dY, AY[c][r]);
        }
    }
}

// The same for random rays: every ray has its own offsets (NRXr, NRYr: minus the ray's offset from the
// tile centre, in both lanes), so neither difference is shared between rays.
template <int C, int R, bool MASS, bool SHARED_RCP>
__device__ __forceinline__ void pair_step_random(const float4 P, const float2 Mm, const float2 (&NRXr)[C][R],
                                                 const float2 (&NRYr)[C][R], float2 (&AX)[C][R], float2 (&AY)[C][R])
{
    const float2 LX = make_float2(P.x, P.y);
    const float2 LY = make_float2(P.z, P.w);
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float2 dX = __fadd2_rn(LX, NRXr[c][r]);
            const float2 dY = __fadd2_rn(LY, NRYr[c][r]);
            const float2 R2 = __ffma2_rn(dY, dY, __fmul2_rn(dX, dX));
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
            AX[c][r] = __ffma2_rn(W, dX, AX[c][r]);
            AY[c][r] = __ffma2_rn(W, dY, AY[c][r]);
        }
    }
}

template <class L, int C, int R, int SHARED4, int FOLD, bool MASS, bool DUMP, bool SPLIT, bool RANDOM = false>
__device__ void tile_fp32(const LaunchArgs &A, const MapDesc &M, unsigned long long tile, int seg, int item,
                          SmemFP32 &S, unsigned &cnt_in, unsigned &cnt_out)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int w = tid >> 5;
    const int col0 = (w % L::WX) * 32 * C + lane;     // column c of this thread: col0 + 32 c
    const int row0 = (w / L::WX) * R;                 // row r: row0 + r
    const long long tx = (long long)(tile % (unsigned long long)M.tiles_x);
    const long long ty = (long long)(tile / (unsigned long long)M.tiles_x);
    const long long ib = M.i0 + tx * kTileX;
    const long long jb = M.j0 + ty * kTileY;

    if (tid == 0) {
        S.cx = ((double)ib + 32.0 - M.half_nx) * M.delta;
        S.cy = ((double)jb + 16.0 - M.half_ny) * M.delta;
    }
    __syncthreads();
    const double cx = S.cx, cy = S.cy;
    const float cxh = __double2float_rn(cx), cxl = __double2float_rn(cx - (double)cxh);
    const float cyh = __double2float_rn(cy), cyl = __double2float_rn(cy - (double)cyh);

    const float dlt = M.delta_f, dll = M.delta_l;
    float2 NRX[C], NRY[R];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float n = (float)(col0 + 32 * c) - 31.5f;
        const float rx = __fmaf_rn(n, dlt, __fmul_rn(n, dll));
        NRX[c] = make_float2(-rx, -rx);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float n = (float)(row0 + r) - 15.5f;
        const float ry = __fmaf_rn(n, dlt, __fmul_rn(n, dll));
        NRY[r] = make_float2(-ry, -ry);
    }
    // random rays: each ray's offset from the tile centre (a random ray stays inside its tile box)
    float2 NRXr[RANDOM ? C : 1][RANDOM ? R : 1], NRYr[RANDOM ? C : 1][RANDOM ? R : 1];
    if constexpr (RANDOM) {
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float fx, fy;
                random_cell(M, ib + col0 + 32 * c, jb + row0 + r, fx, fy);
                const float nx_ = fx - 32.0f, ny_ = fy - 16.0f;      // cells from the centre, exact
                const float rx = __fmaf_rn(nx_, dlt, __fmul_rn(nx_, dll));
                const float ry = __fmaf_rn(ny_, dlt, __fmul_rn(ny_, dll));
                NRXr[c][r] = make_float2(-rx, -rx);
                NRYr[c][r] = make_float2(-ry, -ry);
            }
    }
    const float hx = 32.0f * dlt + kNearRadius;
    const float hy = 16.0f * dlt + kNearRadius;

    // lane partial sums in registers, float-float sums per the layout
    float2 AX[C][R], AY[C][R];
    Sums<C, R, L::SREG, L::NT> acc(S);
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int r = 0; r < R; ++r) {
            AX[c][r] = make_float2(0.f, 0.f);
            AY[c][r] = make_float2(0.f, 0.f);
            acc.set(c, r, make_float4(0.f, 0.f, 0.f, 0.f));
        }
    unsigned onlens = 0;                              // bit c*R + r: ray exactly on a lens

    // lens range of this work item: all lenses, or one segment of a split tile
    const long long lens_begin = SPLIT ? (long long)seg * M.seg_lenses : 0;
    const long long nstar = (SPLIT && M.lens_splits > 1) ? min(M.nstar, lens_begin + M.seg_lenses) : M.nstar;
    for (long long base = lens_begin; base < nstar; base += kChunkLenses) {
        // ---- stage 256 lens pairs relative to the tile centre ----
        __syncthreads();                               // previous chunk fully consumed
#pragma unroll
        for (int t = tid; t < kChunkPairs; t += L::NT) {   // pair t; warps stage whole 32-pair blocks
            const long long la = base + 2 * t;              // lh is padded: la + 1 < padded size
            const bool in_set = MM_BOUNDS(A.check, la + 1 < lens_padded(M.nstar), kChkLensTile);
            const float4 qa = in_set ? M.lh[la] : make_float4(kNullX, 0.f, 0.f, 0.f);
            const float4 qb = in_set ? M.lh[la + 1] : make_float4(kNullX, 0.f, 0.f, 0.f);
            float xa = __fadd_rn(__fsub_rn(qa.x, cxh), __fsub_rn(qa.z, cxl));
            float ya = __fadd_rn(__fsub_rn(qa.y, cyh), __fsub_rn(qa.w, cyl));
            float xb = __fadd_rn(__fsub_rn(qb.x, cxh), __fsub_rn(qb.z, cxl));
            float yb = __fadd_rn(__fsub_rn(qb.y, cyh), __fsub_rn(qb.w, cyl));
            const bool na = fabsf(xa) < hx && fabsf(ya) < hy;
            const bool nb = fabsf(xb) < hx && fabsf(yb) < hy;
            float ma = 1.f, mb = 1.f;
            if (MASS && in_set) {
                ma = M.lmf[la];
                mb = M.lmf[la + 1];
            }
            if (na) { xa = kNullX; ya = 0.f; ma = 0.f; }
            if (nb) { xb = kNullX; yb = 0.f; mb = 0.f; }
            S.pos[t] = make_float4(xa, xb, ya, yb);
            if (MASS) S.mass[t] = make_float2(ma, mb);
            const unsigned ba = __ballot_sync(0xffffffffu, na);
            const unsigned bb = __ballot_sync(0xffffffffu, nb);
            if (lane == 0) {
                S.near_bits[2 * (t >> 5)] = ba;
                S.near_bits[2 * (t >> 5) + 1] = bb;
            }
        }
        __syncthreads();

        // ---- FP32 sweep over the chunk's pairs ----
        const long long left = nstar - base;
        int npairs = (int)((left >= kChunkLenses) ? kChunkPairs : ((left + 1) >> 1));
        npairs = (npairs + 3) & ~3;                    // padded entries are null lenses
        for (int p0 = 0; p0 < npairs; p0 += FOLD) {
            const int pend = min(p0 + FOLD, npairs);
            for (int p = p0; p < pend; p += 4) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float4 P = S.pos[p + u];
                    const float2 Mm = MASS ? S.mass[p + u] : make_float2(1.f, 1.f);
                    if constexpr (RANDOM) {
                        if (u < SHARED4) pair_step_random<C, R, MASS, true>(P, Mm, NRXr, NRYr, AX, AY);
                        else pair_step_random<C, R, MASS, false>(P, Mm, NRXr, NRYr, AX, AY);
                    } else {
                        if (u < SHARED4) pair_step<C, R, MASS, true>(P, Mm, NRX, NRY, AX, AY);
                        else pair_step<C, R, MASS, false>(P, Mm, NRX, NRY, AX, AY);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int r = 0; r < R; ++r) {          // compensated fold of the lane partials
                    float4 a = acc.get(c, r);
                    float s, e;
                    two_sum(a.x, __fadd_rn(AX[c][r].x, AX[c][r].y), s, e);
                    a.x = s;
                    a.y = __fadd_rn(a.y, e);
                    two_sum(a.z, __fadd_rn(AY[c][r].x, AY[c][r].y), s, e);
                    a.z = s;
                    a.w = __fadd_rn(a.w, e);
                    acc.set(c, r, a);
                    AX[c][r] = make_float2(0.f, 0.f);
                    AY[c][r] = make_float2(0.f, 0.f);
                }
        }

        // ---- near lenses of this chunk, in FP64 ----
        unsigned any = 0;
#pragma unroll
        for (int k = 0; k < 2 * kChunkPairs / 32; ++k) any |= S.near_bits[k];
        if (any) {
            for (int k = 0; k < 2 * kChunkPairs / 32; ++k) {
                unsigned bits = S.near_bits[k];
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const long long g = base + 2 * (32 * (k >> 1) + b) + (k & 1);
                    if (!MM_BOUNDS(A.check, g < M.nstar, kChkLensFP64)) continue;
                    const double xl = M.lx[g], yl = M.ly[g];
                    const double ml = MASS ? M.lm[g] : 1.0;
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        double x1 = ((double)(ib + col0 + 32 * c) + 0.5 - M.half_nx) * M.delta;
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            double x2 = ((double)(jb + row0 + r) + 0.5 - M.half_ny) * M.delta;
                            if constexpr (RANDOM) {
                                float fx, fy;
                                random_cell(M, ib + col0 + 32 * c, jb + row0 + r, fx, fy);
                                x1 = random_coord(ib, fx, M.half_nx, M.delta);
                                x2 = random_coord(jb, fy, M.half_ny, M.delta);
                            }
                            const double d1 = xl - x1, d2 = yl - x2;
                            const double r2 = d1 * d1 + d2 * d2;
                            if (r2 == 0.0) {
                                onlens |= 1u << (c * R + r);
                            } else {
                                const double t = ml / r2;
                                float4 a = acc.get(c, r);
                                add_ff(a.x, a.y, t * d1);
                                add_ff(a.z, a.w, t * d2);
                                acc.set(c, r, a);
                            }
                        }
                    }
                }
            }
        }
    }

    // ---- split tile: publish this segment's sums; the last segment combines them ----
    float4 *part = nullptr;
    if (SPLIT && M.lens_splits > 1) {
        part = M.partial + (size_t)tile * (size_t)M.lens_splits * kTileRays;
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float4 a = acc.get(c, r);
                if ((onlens >> (c * R + r)) & 1u) a.x = __int_as_float(0x7fc00000);   // NaN: ray on a lens
                const size_t pi = (size_t)seg * kTileRays + (col0 + 32 * c) + kTileX * (row0 + r);
                if (MM_BOUNDS(A.check, (tile * (size_t)M.lens_splits) * kTileRays + pi <
                                           (size_t)M.tiles_x * (size_t)((M.nj + kTileY - 1) / kTileY) *
                                               (size_t)M.lens_splits * kTileRays,
                               kChkPartial))
                    part[pi] = a;
            }
        __threadfence();
        __syncthreads();
        if (tid == 0)
            S.loop.last_segment =
                MM_BOUNDS(A.check, tile < (unsigned long long)M.tiles_x * (unsigned long long)((M.nj + kTileY - 1) / kTileY),
                          kChkSegDone) &&
                (atomicAdd(M.seg_done + tile, 1u) == (unsigned)(M.lens_splits - 1));
        __syncthreads();
        if (!S.loop.last_segment) return;
        __threadfence();
    }

    // ---- epilogue: lens equation and pixel (float-float) ----
    const float nsf = (float)M.nside;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const long long gi = ib + col0 + 32 * c;
        float uxh, uxl;
        // |2 i + 1 - nx| < 2^23: a 32-bit conversion (the 64-bit one runs on the FP64 pipe), same value
        ff_axis(M.ax_h, M.ax_l, (float)(int)(2 * gi + 1 - M.nx), M.half_n, uxh, uxl);
        const bool col_ok = gi < M.i0 + M.ni;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long gj = jb + row0 + r;
            float uyh, uyl;
            if constexpr (RANDOM) {                       // u = A (2 t0 - n + 2 f) + N/2 per ray
                float fx, fy;
                random_cell(M, gi, gj, fx, fy);
                ff_axis_frac(M.ax_h, M.ax_l, (float)(int)(2 * ib - M.nx), 2.0f * fx, M.half_n, uxh, uxl);
                ff_axis_frac(M.ay_h, M.ay_l, (float)(int)(2 * jb - M.ny), 2.0f * fy, M.half_n, uyh, uyl);
            } else {
                ff_axis(M.ay_h, M.ay_l, (float)(int)(2 * gj + 1 - M.ny), M.half_n, uyh, uyl);
            }
            float4 a;
            if (SPLIT && part) {                          // split tile: segments in order
                const int local = (col0 + 32 * c) + kTileX * (row0 + r);
                a = __ldcg(part + local);
                for (int sg = 1; sg < M.lens_splits; ++sg) a = ff_add4(a, __ldcg(part + (size_t)sg * kTileRays + local));
            } else {
                a = acc.get(c, r);
            }
            const float I1 = ff_pixel(uxh, uxl, a.x, a.y, M.ip_h, M.ip_l);
            const float I2 = ff_pixel(uyh, uyl, a.z, a.w, M.ip_h, M.ip_l);
            const bool valid = col_ok && gj < M.j0 + M.nj;
            const bool inside = valid && !((onlens >> (c * R + r)) & 1u) && I1 >= 0.f && I1 < nsf && I2 >= 0.f &&
                                I2 < nsf;
            const unsigned pix = inside ? (unsigned)I2 * (unsigned)M.nside + (unsigned)I1 : 0xffffffffu;
            emit_ray<DUMP>(A, M, item, (col0 + 32 * c) + kTileX * (row0 + r), valid, inside, pix,
                           -((double)a.x + (double)a.y), -((double)a.z + (double)a.w), cnt_in, cnt_out);
        }
    }
}

template <class L, int C, int R, int SHARED4, int FOLD, bool DUMP, bool SPLIT, bool RANDOM = false>
__device__ __forceinline__ void tile_fp32_any_mass(const LaunchArgs &A, const MapDesc &M, unsigned long long tile,
                                                   int seg, int item, SmemFP32 &S, unsigned &ci, unsigned &co)
{
    if (M.unit_mass) tile_fp32<L, C, R, SHARED4, FOLD, false, DUMP, SPLIT, RANDOM>(A, M, tile, seg, item, S, ci, co);
    else tile_fp32<L, C, R, SHARED4, FOLD, true, DUMP, SPLIT, RANDOM>(A, M, tile, seg, item, S, ci, co);
}

// Runtime variant of a map (shared-reciprocal pairs per 4, fold interval). Random rays take the
// default variant (3 shared pairs of 4, fold every 64 pairs) whatever the map's.
template <class L, int C, int R, bool DUMP, bool SPLIT, bool RANDOM = false>
__device__ void tile_fp32_dispatch(const LaunchArgs &A, const MapDesc &M, unsigned long long tile, int seg,
                                   int item, SmemFP32 &S, unsigned &ci, unsigned &co)
{
    if constexpr (RANDOM) {
        tile_fp32_any_mass<L, C, R, 3, 64, DUMP, SPLIT, true>(A, M, tile, seg, item, S, ci, co);
        return;
    }
    switch (M.variant) {
    case 1: tile_fp32_any_mass<L, C, R, 3, 32, DUMP, SPLIT>(A, M, tile, seg, item, S, ci, co); break;
    case 2: tile_fp32_any_mass<L, C, R, 2, 64, DUMP, SPLIT>(A, M, tile, seg, item, S, ci, co); break;
    case 3: tile_fp32_any_mass<L, C, R, 4, 64, DUMP, SPLIT>(A, M, tile, seg, item, S, ci, co); break;
    default: tile_fp32_any_mass<L, C, R, 3, 64, DUMP, SPLIT>(A, M, tile, seg, item, S, ci, co); break;
    }
}

// SPLIT: the launch contains maps whose tiles are split over lens segments (kept out of
// the kernel used for unsplit launches, whose register allocation it would crowd).
template <int C, int R, bool SREG, int MINB, bool DUMP, bool SPLIT, bool RANDOM = false>
__global__ void __launch_bounds__(Layout<C, R, SREG, MINB>::NT, MINB) k_shoot_fp32(const LaunchArgs A)
{
    using L = Layout<C, R, SREG, MINB>;
    __shared__ SmemFP32 S;
    persistent_loop<DUMP>(A, S.loop, [&](const MapDesc &M, unsigned long long tile, int seg, int item, unsigned &ci,
                                          unsigned &co) {
        tile_fp32_dispatch<L, C, R, DUMP, SPLIT, RANDOM>(A, M, tile, seg, item, S, ci, co);
    });
}

// RANDOM: the kernel for maps of random rays (every map of the launch has MapDesc::random_rays set).
template <int C, int R, bool SREG, int MINB, bool RANDOM = false>
cudaError_t launch_fp32_layout(const LaunchArgs &args, int grid, bool dump, bool split, cudaStream_t s)
{
    constexpr int NT = Layout<C, R, SREG, MINB>::NT;
    if (split) {
        if (dump) k_shoot_fp32<C, R, SREG, MINB, true, true, RANDOM><<<grid, NT, 0, s>>>(args);
        else k_shoot_fp32<C, R, SREG, MINB, false, true, RANDOM><<<grid, NT, 0, s>>>(args);
    } else {
        if (dump) k_shoot_fp32<C, R, SREG, MINB, true, false, RANDOM><<<grid, NT, 0, s>>>(args);
        else k_shoot_fp32<C, R, SREG, MINB, false, false, RANDOM><<<grid, NT, 0, s>>>(args);
    }
    return cudaGetLastError();
}

}  // namespace dev
}  // namespace mm
