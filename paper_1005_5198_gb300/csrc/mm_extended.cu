// mm_extended.cu -- magnification of extended sources: the map convolved with a
// source profile (Sect. 1: "the magnification of an extended source is found by
// convolving a source profile with the magnification map"), and light curves of
// a source moving along a straight track across the convolved map.
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

#include "mm_ctx.h"

namespace mm {
namespace {

// Separable pass: out[j][i] = sum_k g[k] in[j][i + k - h] (dir 0) or in[j + k - h][i] (dir 1);
// NaN where the support leaves the map. Input counts (dir 0, scaled by inv_nrays) or floats.
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

// Disc: direct sum over row spans; span[dj + H] = half-width of the disc on row dj.
__global__ void k_disc(const unsigned *cin, float *out, int n, const int *span, int H, float scale)
{
    const long long total = (long long)n * n;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q % n), j = (int)(q / n);
        if (i - H < 0 || i + H >= n || j - H < 0 || j + H >= n) {
            out[q] = __int_as_float(0x7fc00000);
            continue;
        }
        float s = 0.f;
        for (int dj = -H; dj <= H; ++dj) {
            const int w = span[dj + H];
            const unsigned *row = cin + (long long)(j + dj) * n + i;
            unsigned long long rs = 0;
            for (int di = -w; di <= w; ++di) rs += row[di];
            s += (float)rs;
        }
        out[q] = s * scale;
    }
}

// Bilinear samples of the convolved map at source positions (Einstein radii).
__global__ void k_track(const float *f, int n, double half_side, double pix, double y1a, double y2a, double y1b,
                        double y2b, long long npts, double *mu)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < npts; k += (long long)gridDim.x * blockDim.x) {
        const double t = npts > 1 ? (double)k / (double)(npts - 1) : 0.0;
        const double y1 = y1a + t * (y1b - y1a), y2 = y2a + t * (y2b - y2a);
        const double u = (y1 + half_side) / pix - 0.5, v = (y2 + half_side) / pix - 0.5;
        const double fu = floor(u), fv = floor(v);
        const int i = (int)fu, j = (int)fv;
        if (!(u >= 0.0 && v >= 0.0) || i + 1 >= n || j + 1 >= n) {
            mu[k] = nan("");
            continue;
        }
        const double a = u - fu, b = v - fv;
        const long long q = (long long)j * n + i;
        mu[k] = (1 - a) * (1 - b) * f[q] + a * (1 - b) * f[q + 1] + (1 - a) * b * f[q + n] + a * b * f[q + n + 1];
    }
}

// Convolve map M into the device float buffer dst (n^2). Returns MM_OK or an error.
int convolve(mm_ctx *ctx, const MapObj &M, int profile, double size_re, float *dst, float *tmp, cudaStream_t s)
{
    const int n = M.p.npix_side;
    const double pix = M.g.pix;
    const float inv_nrays = (float)(1.0 / M.p.nrays_per_pix);
    const int grid = std::max(1, std::min(8 * ctx->sms, (int)(((long long)n * n + 255) / 256)));
    cudaError_t e;
    if (profile == MM_PROFILE_GAUSSIAN) {
        const int h = (int)std::ceil(4.0 * size_re / pix);
        std::vector<double> gd(2 * h + 1);
        double tot = 0.0;
        for (int k = -h; k <= h; ++k) tot += gd[k + h] = std::exp(-(k * pix) * (k * pix) / (2.0 * size_re * size_re));
        std::vector<float> g(gd.size());
        for (size_t k = 0; k < gd.size(); ++k) g[k] = (float)(gd[k] / tot);
        float *dg = nullptr;
        int rc = ctx->arena.alloc(g.size() * sizeof(float), (void **)&dg);
        if (rc) return rc;
        if ((e = cudaMemcpyAsync(dg, g.data(), g.size() * sizeof(float), cudaMemcpyHostToDevice, s)) == cudaSuccess) {
            k_gauss_pass<true><<<grid, 256, 0, s>>>(M.counts, nullptr, tmp, n, dg, h, 0, inv_nrays);
            k_gauss_pass<false><<<grid, 256, 0, s>>>(nullptr, tmp, dst, n, dg, h, 1, 1.0f);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        ctx->arena.free(dg);
        return e == cudaSuccess ? MM_OK : cuda_fail(e, "gaussian convolution");
    }
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
    int *ds = nullptr;
    int rc = ctx->arena.alloc(span.size() * sizeof(int), (void **)&ds);
    if (rc) return rc;
    if ((e = cudaMemcpyAsync(ds, span.data(), span.size() * sizeof(int), cudaMemcpyHostToDevice, s)) == cudaSuccess) {
        k_disc<<<grid, 256, 0, s>>>(M.counts, dst, n, ds, H, (float)(1.0 / ((double)taps * M.p.nrays_per_pix)));
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
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
    const size_t npix = (size_t)M->p.npix_side * M->p.npix_side;
    float *buf = nullptr;
    double *dmu = nullptr;
    if ((rc = ctx->arena.alloc(2 * npix * sizeof(float), (void **)&buf))) return rc;
    if ((rc = ctx->arena.alloc((size_t)n_points * sizeof(double), (void **)&dmu))) {
        ctx->arena.free(buf);
        return rc;
    }
    rc = convolve(ctx, *M, profile, size_re, buf, buf + npix, ctx->stream);
    cudaError_t e = cudaSuccess;
    if (!rc) {
        const int grid = (int)std::min<long long>((n_points + 255) / 256, 1024);
        k_track<<<grid, 256, 0, ctx->stream>>>(buf, M->p.npix_side, 0.5 * M->p.side_re, M->g.pix, y1_start, y2_start,
                                                y1_end, y2_end, n_points, dmu);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host_mu, dmu, (size_t)n_points * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    }
    ctx->arena.free(buf);
    ctx->arena.free(dmu);
    if (rc) return rc;
    return e == cudaSuccess ? MM_OK : cuda_fail(e, "light curve");
}
