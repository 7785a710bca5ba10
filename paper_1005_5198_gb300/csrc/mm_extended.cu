// mm_extended.cu -- magnification of extended sources (Sect. 1): a point-source map,
// convolved with the brightness profile of a finite source, gives that source's
// magnification at every position; light curves sample the convolved map along a
// straight track of the source.
//
// Readings where the paper gives no detail:
//   * mu = N / N_rays per pixel; the profile is discretised on the pixel grid and
//     normalised to unit sum;
//   * Gaussian: w(i, j) = g(i) g(j), g(k) = exp(-(k p)^2 / (2 s^2)) for
//     |k| <= h = ceil(4 s / p) (square support, so the convolution is separable);
//   * disc: w(i, j) = 1 for pixel-centre offsets with (i^2 + j^2) p^2 <= R^2;
//   * an output pixel whose profile support leaves the map has no value (NaN);
//   * light curves: bilinear interpolation between pixel centres, which sit at
//     -L/2 + (I + 1/2) p; a sample that needs a pixel without value is NaN.
#include <algorithm>
#include <cmath>
#include <vector>

#include "mm_async.cuh"
#include "mm_ctx.h"

namespace mm {
namespace {

// Separable pass: out[j][i] = sum_k g[k] in[j][i + k - h] (dir 0) or in[j + k - h][i] (dir 1);
// NaN where the support leaves the map. Input counts (scaled by inv_nrays) or floats. Untiled
// maps run dir 1 from the counts, then dir 0.
template <bool FROM_COUNTS>
__global__ void k_gauss_pass(const unsigned *cin, const float *fin, float *out, int n, const float *g, int h, int dir,
                             float inv_nrays)
{
    const long long total = (long long)n * n;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % n), j = (int)(q / n);
        const int c = dir == 0 ? i : j;
        if (c - h < 0 || c + h >= n) {
            out[q] = __int_as_float(0x7fc00000);
            continue;
        }
        float s = 0.f;
        for (int k = -h; k <= h; ++k) {
            const long long src = dir == 0 ? q + k : q + (long long)k * n;
            const float v = FROM_COUNTS ? (float)cin[src] * inv_nrays : fin[src];
            s = fmaf(g[k + h], v, s);
        }
        out[q] = s;
    }
}

// Disc: direct sum over row spans; span[dj + H] = half-width of the disc on row dj. The integer
// total of the disc is converted to float once and scaled by 1 / (taps N_rays).
__global__ void k_disc(const unsigned *cin, float *out, int n, const int *span, int H, float scale)
{
    const long long total = (long long)n * n;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % n), j = (int)(q / n);
        if (i - H < 0 || i + H >= n || j - H < 0 || j + H >= n) {
            out[q] = __int_as_float(0x7fc00000);
            continue;
        }
        unsigned long long total = 0;
        for (int dj = -H; dj <= H; ++dj) {
            const int w = span[dj + H];
            const unsigned *row = cin + (long long)(j + dj) * n + i;
            for (int di = -w; di <= w; ++di) total += row[di];
        }
        out[q] = (float)total * scale;
    }
}

// ---- tiled forms of the passes above: the same per-pixel sums in the same order ----

constexpr int kDiscTileW = 64, kDiscTileH = 64;        // disc: 64 x 64 outputs per CTA
constexpr int kDiscPer = 16;                           // outputs per thread, down its column (4 row groups)
constexpr int kDiscMaxH = 15;                          // widest radius (pixels) of the tiled disc kernel; wider
                                                       // supports take the untiled kernel
constexpr int kGaussMaxTiledH = 131;                   // widest Gaussian half-width of the tiled passes
constexpr size_t kGaussSmemMax = 200 * 1024;           // the Gaussian CTA's shared-memory limit (wider
                                                       // supports take the untiled kernel)

// Gaussian passes (tiled): one kernel, k_gauss_vt, convolves its input down the columns and writes
// the result transposed. Run on the counts it gives V^T, V the column pass; run on V^T it gives the
// row pass of V in the map's own orientation. The two lanes of every packed f32x2 FMA are the same
// output of two neighbouring columns, so one 8-byte shared load gives an operand pair and the taps
// are pairs (g, g). A thread owns 16 consecutive outputs down its pair of columns and runs the taps
// in chunks of 8 (the last one of 4 when TP is not a multiple of 8): per chunk of 8 it loads the 23
// input pairs the 16 outputs need once and makes 128 packed FMAs from them. The taps are padded with
// zero weights to TP, a multiple of 4; a padded tap
// leaves a sum unchanged (0 times a finite input is 0, and every sum is non-negative) or meets only
// an input column that is NaN throughout, whose outputs are NaN anyway. Every output adds its taps
// in order (a correctly rounded FMA each, tap 0 first), exactly as k_gauss_pass. A CTA holds one
// tile, copied in by cp.async (16-byte copies when N_side is a multiple of 4, 4-byte copies
// otherwise); three CTAs per SM hide each other's copies (faster than two double-buffered CTAs).
constexpr int kGOut = 128;                              // outputs per tile down the columns (8 warps x 16)
constexpr int kGPairs = 32;                             // pairs of columns per tile (64 columns), one per lane

__host__ __device__ inline int gauss_taps_padded(int h) { return (2 * h + 1 + 3) & ~3; }
// input rows staged per tile: 128 + TP - 1
__host__ __device__ inline int gauss_span(int h) { return kGOut + gauss_taps_padded(h) - 1; }
__host__ __device__ inline size_t gauss_tile_floats(int h) { return (size_t)2 * kGPairs * gauss_span(h); }
__host__ __device__ inline size_t gauss_smem(int h)
{
    return ((size_t)2 * gauss_taps_padded(h) + gauss_tile_floats(h)) * 4;
}
// Disc tile of radius H: rows [r0 - H, r0 + 64 + H) x columns [c0 - H4, c0 + 64 + H4) of the counts,
// H4 = H rounded up to a multiple of 4 (so that a staged row starts on a 16-byte boundary when N_side
// is a multiple of 4). Shared memory: 32-bit prefix rows [rows x pitch] (pitch = columns + 1, a leading
// zero), then, from the next 16-byte boundary, the raw counts of the next tile [rows x columns]. The
// rare 64-bit prefix rows [rows x pitch] take the bytes of both.
__host__ __device__ constexpr int disc_halo_cols(int H) { return (H + 3) & ~3; }
__host__ __device__ constexpr int disc_cols(int H) { return kDiscTileW + 2 * disc_halo_cols(H); }
__host__ __device__ constexpr int disc_rows(int H) { return kDiscTileH + 2 * H; }
__host__ __device__ constexpr int disc_pitch(int H) { return disc_cols(H) + 1; }
__host__ __device__ constexpr size_t disc_raw_offset(int H)
{
    return ((size_t)disc_rows(H) * disc_pitch(H) * 4 + 15) & ~(size_t)15;
}
__host__ __device__ constexpr size_t disc_smem(int H) { return (size_t)disc_rows(H) * disc_pitch(H) * 8; }
__host__ __device__ constexpr bool disc_layout_fits()
{
    for (int H = 0; H <= kDiscMaxH; ++H)
        if (disc_raw_offset(H) + (size_t)disc_rows(H) * disc_cols(H) * 4 > disc_smem(H) || disc_cols(H) > 96) return false;
    return true;
}
static_assert(disc_layout_fits(), "the raw counts fit beside the 32-bit prefix rows, at most 96 columns");

// CTAs of the tiled disc kernel per SM: as many as its shared memory allows, up to 4 (64 registers).
__host__ __device__ constexpr int disc_ctas_per_sm(int H)
{
    return disc_smem(H) * 4 <= 220 * 1024 ? 4 : disc_smem(H) * 3 <= 220 * 1024 ? 3 : 2;
}

// Row half-widths of a disc, span w[k] on row offset k - H (passed by value to the kernel).
struct DiscSpans {
    int w[2 * kDiscMaxH + 1];
};

// acc[u] = sum over taps k < TP of g[k] x[(u + k) st], u < 16: x the thread's first input pair,
// st the distance between consecutive input pairs (in pairs), gs2 the taps as pairs (g, g).
__device__ __forceinline__ void gauss_taps2(const float2 *gs2, int tp, const float2 *x, int st, float2 (&acc)[16])
{
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] = make_float2(0.f, 0.f);
    int k0 = 0;
    for (; k0 + 8 <= tp; k0 += 8) {
        float2 v[23];
#pragma unroll
        for (int q = 0; q < 23; ++q) v[q] = x[(k0 + q) * st];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const float2 w = gs2[k0 + kk];
#pragma unroll
            for (int u = 0; u < 16; ++u) acc[u] = __ffma2_rn(w, v[u + kk], acc[u]);
        }
    }
    if (k0 < tp) {                                            // the last 4 taps
        float2 v[19];
#pragma unroll
        for (int q = 0; q < 19; ++q) v[q] = x[(k0 + q) * st];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const float2 w = gs2[k0 + kk];
#pragma unroll
            for (int u = 0; u < 16; ++u) acc[u] = __ffma2_rn(w, v[u + kk], acc[u]);
        }
    }
}

// out_t[i][j] = sum_k g[k] in[j + k - h][i] (NaN where j - h < 0 or j + h >= n): a tile is input rows
// [r0 - h, r0 - h + span) of 64 columns [c0, c0 + 64), row-major (zeros outside the map), so that
// columns 2l, 2l + 1 of a row form a pair; lane l takes those two columns, warp w the outputs
// r0 + 16 w .. + 16. Tiles t, t + gridDim.x, ...; each thread copies the same elements of every tile
// and, from counts (mu = N inv_nrays), converts those it copied once they have landed.
template <bool FROM_COUNTS>
__global__ void __launch_bounds__(256, 3) k_gauss_vt(const void *in, float *out_t, int n, const float *g, int h,
                                                     float inv_nrays)
{
    extern __shared__ float4 sm4[];
    const int tp = gauss_taps_padded(h), S = gauss_span(h);
    float2 *const gs2 = reinterpret_cast<float2 *>(sm4);
    float *const tile = reinterpret_cast<float *>(gs2 + tp);
    for (int k = threadIdx.x; k < tp; k += blockDim.x) {       // taps as pairs, zero up to TP
        const float v = k <= 2 * h ? g[k] : 0.f;
        gs2[k] = make_float2(v, v);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int cols = (n + 2 * kGPairs - 1) / (2 * kGPairs), rows = (n + kGOut - 1) / kGOut;
    const long long tiles = (long long)cols * rows;
    const bool vec = (n & 3) == 0;                             // rows start on 16-byte boundaries
    const unsigned *const src_u = static_cast<const unsigned *>(in);
    auto stage = [&](long long t, float *dst) {
        const int c0 = (int)(t % cols) * (2 * kGPairs), r0 = (int)(t / cols) * kGOut;
        if (vec) {
            for (int q = threadIdx.x; q < S * 16; q += blockDim.x) {   // row q / 16, columns 4 (q % 16) ..
                const int j = r0 - h + (q >> 4), i = c0 + 4 * (q & 15);
                const int cnt = (j >= 0 && j < n) ? max(0, min(4, n - i)) : 0;
                cp_async16(dst + 4 * q, src_u + (cnt ? (long long)j * n + i : 0), 4u * cnt);
            }
        } else {
            for (int q = threadIdx.x; q < S * 64; q += blockDim.x) {   // row q / 64, column q % 64
                const int j = r0 - h + (q >> 6), i = c0 + (q & 63);
                const bool ok = j >= 0 && j < n && i < n;
                cp_async4(dst + q, src_u + (ok ? (long long)j * n + i : 0), ok ? 4u : 0u);
            }
        }
        cp_async_commit();
    };
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        stage(t, tile);                                        // the previous tile was released below
        cp_async_wait<0>();
        if (FROM_COUNTS) {                                     // the elements this thread copied, now landed
            if (vec) {
                for (int q = threadIdx.x; q < S * 16; q += blockDim.x) {
                    float4 *const p4 = reinterpret_cast<float4 *>(tile) + q;
                    const uint4 c = *reinterpret_cast<const uint4 *>(p4);
                    *p4 = make_float4((float)c.x * inv_nrays, (float)c.y * inv_nrays, (float)c.z * inv_nrays,
                                      (float)c.w * inv_nrays);
                }
            } else {
                for (int q = threadIdx.x; q < S * 64; q += blockDim.x)
                    tile[q] = (float)__float_as_uint(tile[q]) * inv_nrays;
            }
        }
        __syncthreads();                                       // tile t staged; taps staged
        float2 acc[16];
        gauss_taps2(gs2, tp, reinterpret_cast<const float2 *>(tile) + (w * 16) * kGPairs + lane, kGPairs, acc);
        const int c0 = (int)(t % cols) * (2 * kGPairs), r0 = (int)(t / cols) * kGOut;
        const int j0 = r0 + w * 16;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int i = c0 + 2 * lane + e;
            if (i >= n) continue;
            float v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int j = j0 + u;
                v[u] = (j - h < 0 || j + h >= n) ? __int_as_float(0x7fc00000) : (e ? acc[u].y : acc[u].x);
            }
            float *const o = out_t + (long long)i * n + j0;
            if (vec && j0 + 16 <= n) {
#pragma unroll
                for (int u = 0; u < 16; u += 4) *reinterpret_cast<float4 *>(o + u) = make_float4(v[u], v[u + 1], v[u + 2], v[u + 3]);
            } else {
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    if (j0 + u < n) o[u] = v[u];
            }
        }
        __syncthreads();                                       // every thread has read the tile
    }
}

// Disc (tiled): a CTA stages the counts of its tile with a halo of H rows and H4 columns, and takes
// prefix sums along each staged row (with a leading zero), so the sum over a row span [i - w, i + w]
// is one difference. An output's disc sum is the integer total of its row spans, converted to float
// once (as k_disc). The prefix sums are taken modulo 2^32 first; a CTA-wide vote on the tile's
// largest count picks how the spans are added:
//   every count below 2^32 / (2H + 1)^2: the whole disc sum is below 2^32, so the span
//     differences add up exactly in 32 bits;
//   every count below 2^32 / (2H + 1): each span sum is below 2^32 and its 32-bit difference is
//     exact; the spans add up in 64 bits;
//   otherwise the tile is staged again as 64-bit prefix sums.
// The three ways give the same integer, hence the same float. The kernel is compiled for each radius
// H <= 15: the tap rows and the 16 outputs of a thread are unrolled, so every shared load of a span
// end is an immediate offset from one of two addresses per tap row.

// The raw counts of tile (r0, c0) into raw [rows x columns], zeros outside the map: 16-byte cp.async
// when N_side is a multiple of 4 (a 4-column group is then wholly inside or outside the map), else
// 4-byte copies.
template <int H>
__device__ __forceinline__ void disc_stage(const unsigned *cin, int n, int r0, int c0, bool vec, unsigned *raw)
{
    constexpr int RT = disc_rows(H), CW = disc_cols(H), H4 = disc_halo_cols(H);
    if (vec) {
        constexpr int G = CW / 4;                          // 16-byte groups per row
        for (int q = threadIdx.x; q < RT * G; q += blockDim.x) {
            const int rr = q / G, x = 4 * (q - rr * G);
            const int j = r0 - H + rr, i = c0 - H4 + x;
            const bool ok = j >= 0 && j < n && i >= 0 && i < n;
            cp_async16(raw + rr * CW + x, cin + (ok ? (long long)j * n + i : 0), ok ? 16u : 0u);
        }
    } else {
        for (int q = threadIdx.x; q < RT * CW; q += blockDim.x) {
            const int rr = q / CW, x = q - rr * CW;
            const int j = r0 - H + rr, i = c0 - H4 + x;
            const bool ok = j >= 0 && j < n && i >= 0 && i < n;
            cp_async4(raw + q, cin + (ok ? (long long)j * n + i : 0), ok ? 4u : 0u);
        }
    }
    cp_async_commit();
}

// A tile whose staged rectangle lies inside the map (and N_side a multiple of 4, so that every staged
// row starts on a 16-byte boundary) is staged by one bulk copy per row, completing on bar; warp 0 issues
// them once lane 0 has announced their bytes. Other tiles take disc_stage.
template <int H>
__device__ __forceinline__ bool disc_interior(int n, int r0, int c0)
{
    constexpr int H4 = disc_halo_cols(H);
    return (n & 3) == 0 && r0 - H >= 0 && r0 + kDiscTileH + H <= n && c0 - H4 >= 0 && c0 + kDiscTileW + H4 <= n;
}

template <int H>
__device__ __forceinline__ void disc_stage_bulk(const unsigned *cin, int n, int r0, int c0, unsigned *raw,
                                                uint64_t *bar, bool withhold)
{
    constexpr int RT = disc_rows(H), CW = disc_cols(H), H4 = disc_halo_cols(H);
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0) mbar_arrive_expect(bar, (unsigned)(RT * CW * 4));
        __syncwarp();
        if (!withhold)                                     // (test hook: announce the bytes, copy nothing)
            for (int rr = threadIdx.x; rr < RT; rr += 32)
                bulk_load(raw + rr * CW, cin + (long long)(r0 - H + rr) * n + (c0 - H4), (unsigned)(CW * 4), bar);
    }
}

// 32-bit prefix rows (modulo 2^32, a leading zero) from the staged raw counts: lane l of the row's
// warp adds its three consecutive counts (columns 3l .. 3l + 2; at most 96 columns), then the warp
// scans the lanes' totals. Also the largest count seen, for the CTA's choice of sums.
template <int H>
__device__ __forceinline__ void disc_scan(const unsigned *raw, unsigned *pre, unsigned &maxc)
{
    constexpr int RT = disc_rows(H), CW = disc_cols(H), P = disc_pitch(H);
    static_assert(CW <= 96, "three columns per lane");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int rr = warp; rr < RT; rr += 8) {                // unrolled: the rows' shuffle scans overlap
        const unsigned *const r = raw + rr * CW;
        unsigned *const p = pre + rr * P;
        const int x = 3 * lane;
        const unsigned a0 = x < CW ? r[x] : 0u, a1 = x + 1 < CW ? r[x + 1] : 0u, a2 = x + 2 < CW ? r[x + 2] : 0u;
        maxc = max(maxc, max(a0, max(a1, a2)));
        const unsigned s0 = a0, s1 = a0 + a1, s2 = s1 + a2;
        unsigned incl = s2;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        const unsigned excl = incl - s2;
        if (lane == 0) p[0] = 0u;
        if (x < CW) p[x + 1] = excl + s0;
        if (x + 1 < CW) p[x + 2] = excl + s1;
        if (x + 2 < CW) p[x + 3] = excl + s2;
    }
}

// 64-bit prefix rows of tile (r0, c0) read from global memory (the rare tiles with a count of
// 2^32 / (2H + 1) or more); one warp per row.
__device__ __forceinline__ void disc_prefix64(const unsigned *cin, int n, int r0, int c0, int H, unsigned long long *pre)
{
    const int RT = disc_rows(H), CW = disc_cols(H), P = disc_pitch(H), H4 = disc_halo_cols(H);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
    for (int rr = warp; rr < RT; rr += 8) {
        const int j = r0 - H + rr;
        unsigned long long carry = 0;
        if (lane == 0) pre[rr * P] = 0;
#pragma unroll 1
        for (int x0 = 0; x0 < CW; x0 += 32) {
            const int x = x0 + lane, i = c0 - H4 + x;
            const unsigned cnt = (x < CW && j >= 0 && j < n && i >= 0 && i < n) ? cin[(long long)j * n + i] : 0u;
            unsigned long long v = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            if (x < CW) pre[rr * P + x + 1] = carry + v;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
}

// Thread (column c, row group g) computes outputs r0 + 16 g + u, u < 16, of column c0 + c: for tap row
// k (row offset k - H) and output u the staged row is 16 g + u + k, and the span of half-width w[k]
// is pre[.. + w + 1] - pre[.. - w]. PT: prefix type; A: accumulator type. The integer totals go out
// as floats, NaN where the disc leaves the map.
template <typename A>
__device__ __forceinline__ void disc_store(const A (&acc)[kDiscPer], float *out, int n, int r0, int c0, int H,
                                           float scale)
{
    const int c = threadIdx.x & (kDiscTileW - 1), g = threadIdx.x / kDiscTileW;
    const int i = c0 + c;
    const bool col_ok = i - H >= 0 && i + H < n;
#pragma unroll
    for (int u = 0; u < kDiscPer; ++u) {
        const int j = r0 + kDiscPer * g + u;
        if (i < n && j < n)
            out[(long long)j * n + i] = (col_ok && j - H >= 0 && j + H < n) ? (float)acc[u] * scale
                                                                            : __int_as_float(0x7fc00000);
    }
}

// The common way (32-bit prefix rows and sums), compiled for each radius: the tap rows and the 16
// outputs unrolled, so that every load is an immediate offset from base (the thread's column on its
// first staged row) plus the tap row's span end, which is the same for every thread of the launch.
// Tap rows k and 2H - k have the same span, so the two span ends loaded on staged row r serve output
// r - k and output r - (2H - k) alike: 27 instead of 34 loads per output at H = 8.
template <int H>
__device__ __forceinline__ void disc_outputs32(const unsigned *base, const DiscSpans &sp, float *out, int n, int r0,
                                               int c0, float scale)
{
    constexpr int P = disc_pitch(H);
    unsigned acc[kDiscPer];
#pragma unroll
    for (int u = 0; u < kDiscPer; ++u) acc[u] = 0u;
#pragma unroll
    for (int k = 0; k <= H; ++k) {
        const int km = 2 * H - k;                          // the mirrored tap row
        const unsigned *const hi = base + sp.w[k] + 1, *const lo = base - sp.w[k];
#pragma unroll
        for (int r = k; r < kDiscPer + km; ++r) {          // staged rows of output r - k or r - km
            const bool first = r - k < kDiscPer, second = km != k && r - km >= 0;
            if (!first && !second) continue;
            const unsigned span = hi[r * P] - lo[r * P];
            if (first) acc[r - k] += span;
            if (second) acc[r - km] += span;
        }
    }
    disc_store<unsigned>(acc, out, n, r0, c0, H, scale);
}

// The rare ways (64-bit sums of 32-bit spans, or 64-bit prefix rows): the same sums, tap rows not
// unrolled.
template <typename PT>
__device__ __forceinline__ void disc_outputs64(const PT *pre, const int *sp, float *out, int n, int r0, int c0,
                                            int H, float scale)
{
    const int P = disc_pitch(H), H4 = disc_halo_cols(H);
    const int c = threadIdx.x & (kDiscTileW - 1), g = threadIdx.x / kDiscTileW;
    const PT *const base = pre + (kDiscPer * g) * P + c + H4;
    unsigned long long acc[kDiscPer];
#pragma unroll
    for (int u = 0; u < kDiscPer; ++u) acc[u] = 0ull;
#pragma unroll 1
    for (int k = 0; k <= 2 * H; ++k) {
        const int w = sp[k];
        const PT *const hi = base + k * P + w + 1, *const lo = base + k * P - w;
#pragma unroll
        for (int u = 0; u < kDiscPer; ++u) acc[u] += (unsigned long long)(PT)(hi[u * P] - lo[u * P]);
    }
    disc_store<unsigned long long>(acc, out, n, r0, c0, H, scale);
}

// A CTA takes tiles t, t + gridDim.x, ...: while it computes the outputs of one tile, the raw counts of
// the next arrive (bulk copies for interior tiles, cp.async otherwise). A 64-bit tile (rare) waits for
// its outputs before the next copy starts, since its prefix rows cover the staging buffer. A wait for
// bulk copies that runs out of time sets *fault and ends the CTA.
template <int H>
__global__ void __launch_bounds__(256, disc_ctas_per_sm(H)) k_disc_tiled(const unsigned *cin, float *out, int n,
                                                                         const DiscSpans sp, float scale,
                                                                         unsigned *fault, int withhold)
{
    extern __shared__ uint4 dsm[];
    __shared__ int spans[2 * H + 1];                       // the spans, read by index in the 64-bit ways
    __shared__ uint64_t bar;                               // completion of a tile's bulk copies
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k <= 2 * H; ++k) spans[k] = sp.w[k];
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    unsigned *const pre32 = reinterpret_cast<unsigned *>(dsm);
    unsigned long long *const pre64 = reinterpret_cast<unsigned long long *>(dsm);
    unsigned *const raw = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(dsm) + disc_raw_offset(H));
    // this thread's column on its first staged row (the same for every tile)
    const unsigned *const base = pre32 + (kDiscPer * (threadIdx.x / kDiscTileW)) * disc_pitch(H) +
                                 (threadIdx.x & (kDiscTileW - 1)) + disc_halo_cols(H);
    const bool vec = (n & 3) == 0;
    const int cols = (n + kDiscTileW - 1) / kDiscTileW, rows = (n + kDiscTileH - 1) / kDiscTileH;
    const long long tiles = (long long)cols * rows;
    const unsigned long long taps1 = (unsigned long long)(2 * H + 1);
    const unsigned small_span = (unsigned)(0xffffffffull / taps1);             // span sums below 2^32
    const unsigned small_disc = (unsigned)(0xffffffffull / (taps1 * taps1));   // disc sums below 2^32
    auto stage = [&](long long t) {
        const int c0 = (int)(t % cols) * kDiscTileW, r0 = (int)(t / cols) * kDiscTileH;
        if (disc_interior<H>(n, r0, c0)) disc_stage_bulk<H>(cin, n, r0, c0, raw, &bar, withhold != 0);
        else disc_stage<H>(cin, n, r0, c0, vec, raw);
    };
    unsigned phase = 0u;
    if (blockIdx.x < tiles) stage(blockIdx.x);
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int c0 = (int)(t % cols) * kDiscTileW, r0 = (int)(t / cols) * kDiscTileH;
        if (disc_interior<H>(n, r0, c0)) {
            const bool ok = mbar_wait(&bar, phase);
            if (__syncthreads_or(!ok)) {                   // (also the barrier below)
                if (threadIdx.x == 0) {
                    atomicExch(fault, 1u);
                    mbar_wait(&bar, phase);                // copies still in flight land before the CTA ends
                }
                return;
            }
            phase ^= 1u;
        } else {
            cp_async_wait<0>();
            __syncthreads();                               // tile t's counts staged; the previous outputs done
        }
        unsigned maxc = 0;
        disc_scan<H>(raw, pre32, maxc);
        // (both votes are also barriers: the raw counts are read and the prefix rows written)
        const bool not_disc32 = __syncthreads_or(maxc >= small_disc), not_span32 = __syncthreads_or(maxc >= small_span);
        const long long tn = t + gridDim.x;
        if (!not_span32) {
            if (tn < tiles) stage(tn);
            if (!not_disc32) disc_outputs32<H>(base, sp, out, n, r0, c0, scale);
            else disc_outputs64<unsigned>(pre32, spans, out, n, r0, c0, H, scale);
        } else {                                           // a count of 2^32 / (2H + 1) or more: 64 bits
            disc_prefix64(cin, n, r0, c0, H, pre64);
            __syncthreads();
            disc_outputs64<unsigned long long>(pre64, spans, out, n, r0, c0, H, scale);
            __syncthreads();                               // the prefix rows over the staging buffer are read
            if (tn < tiles) stage(tn);
        }
    }
}

using DiscKernel = void (*)(const unsigned *, float *, int, const DiscSpans, float, unsigned *, int);
template <int... Hs>
struct DiscKernels {
    static constexpr DiscKernel table[] = {k_disc_tiled<Hs>...};
};
static_assert(kDiscMaxH == 15, "the kernel table lists H = 0 .. 15");
using DiscTable = DiscKernels<0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15>;

// Sample k of a light curve: t = k / (npts - 1) along the track, the pixel (i, j) below and left of
// the sample (pixel centres at -L/2 + (I + 1/2) p) and the bilinear weights (a, b). False where the
// sample needs a pixel outside the map (tested in FP64, before any conversion to int).
__device__ __forceinline__ bool lc_sample(long long k, long long npts, int n, double half_side, double pix, double y1a,
                                          double y2a, double y1b, double y2b, int &i, int &j, double &a, double &b)
{
    const double t = npts > 1 ? (double)k / (double)(npts - 1) : 0.0;
    const double y1 = y1a + t * (y1b - y1a), y2 = y2a + t * (y2b - y2a);
    const double u = (y1 + half_side) / pix - 0.5, v = (y2 + half_side) / pix - 0.5;
    const double fu = floor(u), fv = floor(v);
    if (!(u >= 0.0 && v >= 0.0) || !(fu + 1.0 < (double)n) || !(fv + 1.0 < (double)n)) return false;
    i = (int)fu;
    j = (int)fv;
    a = u - fu;
    b = v - fv;
    return true;
}

// The bilinear interpolation of the four pixels (i, j), (i + 1, j), (i, j + 1), (i + 1, j + 1); one
// function for every light-curve kernel, so that equal pixels give equal samples.
__device__ __forceinline__ double lc_bilinear(double a, double b, float f00, float f10, float f01, float f11)
{
    return (1 - a) * (1 - b) * f00 + a * (1 - b) * f10 + (1 - a) * b * f01 + a * b * f11;
}

// Bilinear samples of the convolved map at source positions (Einstein radii).
__global__ void k_track(const float *f, int n, double half_side, double pix, double y1a, double y2a, double y1b,
                        double y2b, long long npts, double *mu)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < npts; k += (long long)gridDim.x * blockDim.x) {
        int i, j;
        double a, b;
        if (!lc_sample(k, npts, n, half_side, pix, y1a, y2a, y1b, y2b, i, j, a, b)) {
            mu[k] = nan("");
            continue;
        }
        const long long q = (long long)j * n + i;
        mu[k] = lc_bilinear(a, b, f[q], f[q + 1], f[q + n], f[q + n + 1]);
    }
}

// ---- light curves without the whole convolved map ----
// A light curve needs the convolved map at four pixels per sample only. When that is less work than
// convolving the map, a CTA per sample computes its four pixels directly, with the same arithmetic as
// the passes above, so that every pixel, and hence every sample, equals what sampling the convolved
// map gives, bit for bit.

constexpr int kLcChunk = 256;                           // column sums per row and round (Gaussian)
constexpr int kLcTaps = 2048;                           // taps held in shared memory (wider Gaussians read
                                                        // them from global memory)

// Gaussian: for rows j and j + 1 the column sums V[r][x] = sum_k g[k] mu[j + r + k - h][x] (FMA chain in
// tap order, as the column pass) over the columns the row sums need, in rounds of kLcChunk + 1
// columns; then thread o < 4 extends the row sum of pixel (i + (o & 1), j + (o >> 1)) over the round's
// taps (FMA chain in tap order, as the row pass). The taps sit in shared memory (up to kLcTaps of
// them) and the chains are unrolled, so that their loads are issued ahead of the FMAs. A pixel whose
// support leaves the map is NaN.
__global__ void __launch_bounds__(256) k_track_gauss(const unsigned *cin, int n, const float *g, int h, float inv_nrays,
                                                     double half_side, double pix, double y1a, double y2a, double y1b,
                                                     double y2b, long long npts, double *mu)
{
    __shared__ float V[2][kLcChunk + 1];
    __shared__ float gsh[kLcTaps];
    __shared__ float f[4];
    const int T = 2 * h + 1, o = threadIdx.x;
    if (T <= kLcTaps)
        for (int k = o; k < T; k += blockDim.x) gsh[k] = g[k];
    __syncthreads();
    const float *const gt = T <= kLcTaps ? gsh : g;
    for (long long k = blockIdx.x; k < npts; k += gridDim.x) {
        int i, j;
        double a, b;
        if (!lc_sample(k, npts, n, half_side, pix, y1a, y2a, y1b, y2b, i, j, a, b)) {   // the same for the CTA
            if (o == 0) mu[k] = nan("");
            continue;
        }
        const int I = i + (o & 1), J = j + (o >> 1);
        const bool valid = o < 4 && I - h >= 0 && I + h < n && J - h >= 0 && J + h < n;
        float s = 0.f;
        for (int c0 = 0; c0 < T; c0 += kLcChunk) {
            for (int q = o; q < 2 * (kLcChunk + 1); q += blockDim.x) {
                const int r = q / (kLcChunk + 1), t = q - r * (kLcChunk + 1);
                const int x = i - h + c0 + t, row = j + r;
                float v = 0.f;
                if (c0 + t <= T && x >= 0 && x < n && row - h >= 0 && row + h < n) {
                    const unsigned *col = cin + (long long)(row - h) * n + x;
#pragma unroll 16
                    for (int kk = 0; kk < T; ++kk) v = fmaf(gt[kk], __fmul_rn((float)col[(long long)kk * n], inv_nrays), v);
                }
                V[r][t] = v;
            }
            __syncthreads();
            if (valid) {
                const int end = min(T, c0 + kLcChunk);
#pragma unroll 16
                for (int kk = c0; kk < end; ++kk) s = fmaf(gt[kk], V[o >> 1][(o & 1) + kk - c0], s);
            }
            __syncthreads();
        }
        if (o < 4) f[o] = valid ? s : __int_as_float(0x7fc00000);
        __syncthreads();
        if (o == 0) mu[k] = lc_bilinear(a, b, f[0], f[1], f[2], f[3]);
        __syncthreads();
    }
}

// Disc: the integer totals of the four pixels' discs (warp w takes staged rows w, w + 8, ... of rows
// j - H .. j + 1 + H, its lanes the columns), reduced exactly and converted to float once, as the
// disc kernels do. span[dj + H] = half-width of the disc on row offset dj.
__global__ void __launch_bounds__(256) k_track_disc(const unsigned *cin, int n, const int *span, int H, float scale,
                                                    double half_side, double pix, double y1a, double y2a, double y1b,
                                                    double y2b, long long npts, double *mu)
{
    __shared__ unsigned long long tot[8][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long k = blockIdx.x; k < npts; k += gridDim.x) {
        int i, j;
        double a, b;
        if (!lc_sample(k, npts, n, half_side, pix, y1a, y2a, y1b, y2b, i, j, a, b)) {
            if (threadIdx.x == 0) mu[k] = nan("");
            continue;
        }
        unsigned long long p[4] = {0ull, 0ull, 0ull, 0ull};   // pixels (i, j), (i + 1, j), (i, j + 1), (i + 1, j + 1)
        for (int rr = warp; rr < 2 * H + 2; rr += 8) {
            const int row = j - H + rr;
            if (row < 0 || row >= n) continue;
            const int d0 = rr - H, d1 = rr - H - 1;          // row offset from j and from j + 1
            const int w0 = d0 <= H ? span[d0 + H] : -1, w1 = d1 >= -H ? span[d1 + H] : -1;
            const int wm = max(w0, w1);
            const unsigned *const r = cin + (long long)row * n;
            for (int dx = -wm + lane; dx <= wm + 1; dx += 32) {
                const int x = i + dx;
                if (x < 0 || x >= n) continue;
                const unsigned long long c = r[x];
                if (dx >= -w0 && dx <= w0) p[0] += c;
                if (dx - 1 >= -w0 && dx - 1 <= w0) p[1] += c;
                if (dx >= -w1 && dx <= w1) p[2] += c;
                if (dx - 1 >= -w1 && dx - 1 <= w1) p[3] += c;
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) p[e] += __shfl_down_sync(0xffffffffu, p[e], off);
            if (lane == 0) tot[warp][e] = p[e];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float fv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                unsigned long long t = 0;
                for (int w = 0; w < 8; ++w) t += tot[w][e];
                const int I = i + (e & 1), J = j + (e >> 1);
                fv[e] = (I - H >= 0 && I + H < n && J - H >= 0 && J + H < n) ? (float)t * scale
                                                                            : __int_as_float(0x7fc00000);
            }
            mu[k] = lc_bilinear(a, b, fv[0], fv[1], fv[2], fv[3]);
        }
        __syncthreads();
    }
}

// The Gaussian's normalised taps g[0 .. 2h] (FP64, rounded to float once), h = ceil(4 s / p).
std::vector<float> gauss_taps(double size_re, double pix, int *h_out)
{
    const int h = (int)std::ceil(4.0 * size_re / pix);
    std::vector<double> gd(2 * h + 1);
    double tot = 0.0;
    for (int k = -h; k <= h; ++k) tot += gd[k + h] = std::exp(-(k * pix) * (k * pix) / (2.0 * size_re * size_re));
    std::vector<float> g(gd.size());
    for (size_t k = 0; k < gd.size(); ++k) g[k] = (float)(gd[k] / tot);
    *h_out = h;
    return g;
}

// The disc's row half-widths span[dj + H], H = floor(R / p), and its pixel count.
std::vector<int> disc_spans(double size_re, double pix, int *H_out, long long *taps_out)
{
    const double rp = size_re / pix;
    const int H = (int)std::floor(rp);
    std::vector<int> span(2 * H + 1);
    long long taps = 0;
    for (int dj = -H; dj <= H; ++dj) {
        int w = 0;
        while ((double)(w + 1) * (w + 1) + (double)dj * dj <= rp * rp) ++w;
        span[dj + H] = w;
        taps += 2 * w + 1;
    }
    *H_out = H;
    *taps_out = taps;
    return span;
}

// The device time between ctx->ev0 and ctx->ev1 (both recorded and complete) becomes the context's
// last kernel time, over `launches` kernels.
void note_kernel_time(mm_ctx *ctx, int launches)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1) == cudaSuccess) {
        ctx->last_ms = ms;
        ctx->last_launches = launches;
    }
}

// Convolve map M into the device float buffer dst (n^2) on stream s and wait for it; the convolution
// kernels are bracketed by the context's events (note_kernel_time). Returns MM_OK or an error.
int convolve(mm_ctx *ctx, const MapObj &M, int profile, double size_re, float *dst, float *tmp, cudaStream_t s)
{
    const int n = M.p.npix_side;
    const double pix = M.g.pix;
    const float inv_nrays = (float)(1.0 / M.p.nrays_per_pix);
    const int grid = std::max(1, std::min(8 * ctx->sms, (int)(((long long)n * n + 255) / 256)));
    cudaError_t e;
    if (profile == MM_PROFILE_GAUSSIAN) {
        int h = 0;
        const std::vector<float> g = gauss_taps(size_re, pix, &h);
        float *dg = nullptr;
        int rc = ctx->arena.alloc(g.size() * sizeof(float), (void **)&dg);
        if (rc) return rc;
        if ((e = cudaMemcpyAsync(dg, g.data(), g.size() * sizeof(float), cudaMemcpyHostToDevice, s)) == cudaSuccess) {
            const size_t smem = gauss_smem(h);
            // tiled passes: as many CTAs as fit the SMs at once (each loops over its tiles); the
            // column pass from the counts, written transposed, then the same kernel on it
            const long long tiles = (long long)((n + 2 * kGPairs - 1) / (2 * kGPairs)) * ((n + kGOut - 1) / kGOut);
            auto resident = [&](const void *fn) {
                int per_sm = 1;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem) != cudaSuccess) per_sm = 1;
                return (int)std::max(1LL, std::min(tiles, (long long)std::max(1, per_sm) * ctx->sms));
            };
            if (h <= kGaussMaxTiledH) {
                const void *f1 = (const void *)k_gauss_vt<true>, *f2 = (const void *)k_gauss_vt<false>;
                if ((e = cudaFuncSetAttribute(f1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGaussSmemMax)) ==
                        cudaSuccess &&
                    (e = cudaFuncSetAttribute(f2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGaussSmemMax)) ==
                        cudaSuccess) {
                    cudaEventRecord(ctx->ev0, s);
                    k_gauss_vt<true><<<resident(f1), 256, smem, s>>>(M.counts, tmp, n, dg, h, inv_nrays);
                    k_gauss_vt<false><<<resident(f2), 256, smem, s>>>(tmp, dst, n, dg, h, 1.0f);
                    cudaEventRecord(ctx->ev1, s);
                }
            } else {                                           // the same sums: columns, then rows
                cudaEventRecord(ctx->ev0, s);
                k_gauss_pass<true><<<grid, 256, 0, s>>>(M.counts, nullptr, tmp, n, dg, h, 1, inv_nrays);
                k_gauss_pass<false><<<grid, 256, 0, s>>>(nullptr, tmp, dst, n, dg, h, 0, 1.0f);
                cudaEventRecord(ctx->ev1, s);
            }
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e == cudaSuccess) note_kernel_time(ctx, 2);
        }
        ctx->arena.free(dg);
        return e == cudaSuccess ? MM_OK : cuda_fail(e, "gaussian convolution");
    }
    int H = 0;
    long long taps = 0;
    const std::vector<int> span = disc_spans(size_re, pix, &H, &taps);
    const float scale = (float)(1.0 / ((double)taps * M.p.nrays_per_pix));
    if (H <= kDiscMaxH) {                                  // tiled: the kernel compiled for this radius
        DiscSpans sp{};
        for (int k = 0; k <= 2 * H; ++k) sp.w[k] = span[k];
        const DiscKernel fn = DiscTable::table[H];
        const size_t smem = disc_smem(H);
        e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem) != cudaSuccess) per_sm = 1;
        const long long tiles = (long long)((n + kDiscTileW - 1) / kDiscTileW) * ((n + kDiscTileH - 1) / kDiscTileH);
        const int dgrid = (int)std::max(1LL, std::min(tiles, (long long)std::max(1, per_sm) * ctx->sms));
        unsigned *dfault = nullptr, hfault = 0;
        int rc = ctx->arena.alloc(sizeof(unsigned), (void **)&dfault);
        if (rc) return rc;
        const int withhold = take_injection(ctx, MM_INJECT_DISC_NO_COPY) ? 1 : 0;
        if (e == cudaSuccess) e = cudaMemsetAsync(dfault, 0, sizeof(unsigned), s);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev0, s);
        if (e == cudaSuccess) fn<<<dgrid, 256, smem, s>>>(M.counts, dst, n, sp, scale, dfault, withhold);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev1, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hfault, dfault, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) note_kernel_time(ctx, 1);
        ctx->arena.free(dfault);
        if (e != cudaSuccess) return cuda_fail(e, "disc convolution");
        return hfault ? fail(MM_EDEVICE, "k_disc_tiled: a copy into shared memory did not complete") : MM_OK;
    }
    int *ds = nullptr;
    int rc = ctx->arena.alloc(span.size() * sizeof(int), (void **)&ds);
    if (rc) return rc;
    if ((e = cudaMemcpyAsync(ds, span.data(), span.size() * sizeof(int), cudaMemcpyHostToDevice, s)) == cudaSuccess) {
        cudaEventRecord(ctx->ev0, s);
        k_disc<<<grid, 256, 0, s>>>(M.counts, dst, n, ds, H, scale);
        cudaEventRecord(ctx->ev1, s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) note_kernel_time(ctx, 1);
    }
    ctx->arena.free(ds);
    return e == cudaSuccess ? MM_OK : cuda_fail(e, "disc convolution");
}

int prepare(mm_ctx *ctx, mm_map map, int profile, double size_re, std::shared_ptr<MapObj> *out)
{
    if (!ctx) return fail(MM_EINVAL, "null context");
    if (profile != MM_PROFILE_GAUSSIAN && profile != MM_PROFILE_DISC) return fail(MM_EINVAL, "bad profile");
    std::shared_ptr<MapObj> M;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->maps.find(map);
        if (it == ctx->maps.end()) return fail(MM_ENOTFOUND, "unknown map");
        M = it->second;
    }
    if (!(size_re > 0.0) || !std::isfinite(size_re)) return fail(MM_EINVAL, "source size must be > 0");
    const double reach = (profile == MM_PROFILE_GAUSSIAN ? 4.0 : 1.0) * size_re / M->g.pix;
    if (2.0 * reach + 1.0 > (double)M->p.npix_side) return fail(MM_EINVAL, "source profile wider than the map");
    cudaSetDevice(ctx->device);
    const cudaError_t e = cudaStreamWaitEvent(ctx->stream, M->done, 0);
    if (e != cudaSuccess) return cuda_fail(e, "wait for map");
    *out = M;
    return MM_OK;
}

}  // namespace
}  // namespace mm

using namespace mm;

extern "C" int mm_map_convolve(mm_ctx *ctx, mm_map map, int32_t profile, double size_re, float *host_mu,
                               size_t n_elems)
{
    std::shared_ptr<MapObj> M;
    int rc = prepare(ctx, map, profile, size_re, &M);
    if (rc) return rc;
    const size_t npix = (size_t)M->p.npix_side * M->p.npix_side;
    if (!host_mu || n_elems != npix) return fail(MM_EINVAL, "host buffer must hold N_side^2 floats");
    float *buf = nullptr;
    if ((rc = ctx->arena.alloc(2 * npix * sizeof(float), (void **)&buf))) return rc;
    rc = convolve(ctx, *M, profile, size_re, buf, buf + npix, ctx->stream);
    cudaError_t e = cudaSuccess;
    if (!rc) {
        e = cudaMemcpyAsync(host_mu, buf, npix * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    }
    ctx->arena.free(buf);
    if (rc) return rc;
    return e == cudaSuccess ? MM_OK : cuda_fail(e, "convolved map readback");
}

extern "C" int mm_map_lightcurve(mm_ctx *ctx, mm_map map, int32_t profile, double size_re, double y1_start,
                                 double y2_start, double y1_end, double y2_end, int64_t n_points, double *host_mu)
{
    std::shared_ptr<MapObj> M;
    int rc = prepare(ctx, map, profile, size_re, &M);
    if (rc) return rc;
    if (n_points <= 0 || !host_mu) return fail(MM_EINVAL, "need n_points > 0 and an output buffer");
    const int n = M->p.npix_side;
    const size_t npix = (size_t)n * n;
    const double pix = M->g.pix, half = 0.5 * M->p.side_re;
    cudaStream_t s = ctx->stream;
    // Work of the two routes, in operations per light curve: four pixels per sample (the Gaussian's
    // column sums of two rows, 2 (T + 1) T, and four row sums, 4 T; the disc's four pixel totals) or
    // the whole convolution (2 T per pixel for the Gaussian; 2 (2H + 1) span ends per pixel for the
    // tiled disc, its pixel count for the untiled one).
    int h = 0, H = 0;
    long long taps = 0;
    std::vector<float> g;
    std::vector<int> span;
    double local_ops, full_ops;
    if (profile == MM_PROFILE_GAUSSIAN) {
        g = gauss_taps(size_re, pix, &h);
        const double T = 2.0 * h + 1.0;
        local_ops = (double)n_points * (2.0 * (T + 1.0) * T + 4.0 * T);
        full_ops = (double)npix * 2.0 * T;
    } else {
        span = disc_spans(size_re, pix, &H, &taps);
        local_ops = (double)n_points * 4.0 * (double)taps;
        full_ops = (double)npix * (H <= kDiscMaxH ? 2.0 * (2 * H + 1) : (double)taps);
    }
    double *dmu = nullptr;
    if ((rc = ctx->arena.alloc((size_t)n_points * sizeof(double), (void **)&dmu))) return rc;
    cudaError_t e = cudaSuccess;
    const int grid = (int)std::min<long long>(n_points, 64LL * ctx->sms);
    if (local_ops <= full_ops) {                           // a CTA per sample: its four pixels only
        void *dw = nullptr;
        const size_t wbytes = profile == MM_PROFILE_GAUSSIAN ? g.size() * sizeof(float) : span.size() * sizeof(int);
        if ((rc = ctx->arena.alloc(wbytes, &dw))) {
            ctx->arena.free(dmu);
            return rc;
        }
        const void *src = profile == MM_PROFILE_GAUSSIAN ? (const void *)g.data() : (const void *)span.data();
        e = cudaMemcpyAsync(dw, src, wbytes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev0, s);
        if (e == cudaSuccess) {
            if (profile == MM_PROFILE_GAUSSIAN)
                k_track_gauss<<<grid, 256, 0, s>>>(M->counts, n, (const float *)dw, h, (float)(1.0 / M->p.nrays_per_pix),
                                                   half, pix, y1_start, y2_start, y1_end, y2_end, n_points, dmu);
            else
                k_track_disc<<<grid, 256, 0, s>>>(M->counts, n, (const int *)dw, H,
                                                  (float)(1.0 / ((double)taps * M->p.nrays_per_pix)), half, pix, y1_start,
                                                  y2_start, y1_end, y2_end, n_points, dmu);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev1, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host_mu, dmu, (size_t)n_points * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) note_kernel_time(ctx, 1);
        ctx->arena.free(dw);
        ctx->arena.free(dmu);
        return e == cudaSuccess ? MM_OK : cuda_fail(e, "light curve");
    }
    float *buf = nullptr;                                  // the whole convolved map, then samples of it
    if ((rc = ctx->arena.alloc(2 * npix * sizeof(float), (void **)&buf))) {
        ctx->arena.free(dmu);
        return rc;
    }
    rc = convolve(ctx, *M, profile, size_re, buf, buf + npix, s);
    if (!rc) {
        k_track<<<(int)std::min<long long>((n_points + 255) / 256, 1024), 256, 0, s>>>(buf, n, half, pix, y1_start,
                                                                                      y2_start, y1_end, y2_end,
                                                                                      n_points, dmu);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host_mu, dmu, (size_t)n_points * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    ctx->arena.free(buf);
    ctx->arena.free(dmu);
    if (rc) return rc;
    return e == cudaSuccess ? MM_OK : cuda_fail(e, "light curve");
}
