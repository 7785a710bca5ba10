// mm_stats.cu -- statistical comparison of two magnification maps on the device
// (Sect. 3.1: RMS difference of the maps in magnitudes, and a two-sample
// Kolmogorov-Smirnov test on the distributions of Delta m, Eq. deltam).
//
// Delta m_ij = -2.5 log10(mu_ij), mu_ij = N_ij / N_rays. Readings where the
// paper is silent:
//   * RMS: over the pixels where both maps count at least one ray (Delta m of an
//     empty pixel is +infinity); the number of such pixels is reported;
//   * K-S: empty pixels take Delta m = +infinity. Delta m is strictly decreasing in
//     mu, so the K-S statistic of the Delta m samples is the supremum over mu of
//     |P(mu_a >= mu) - P(mu_b >= mu)|, attained at sample values; it is computed
//     exactly from the two count histograms (survivor counts at every value
//     k / N_rays present in either map);
//   * probability: the asymptotic Kolmogorov distribution,
//     Q(l) = 2 sum_{j>=1} (-1)^(j-1) exp(-2 j^2 l^2), at
//     l = (sqrt(n_e) + 0.12 + 0.11 / sqrt(n_e)) D, n_e = n_a n_b / (n_a + n_b)
//     (Stephens' small-sample correction).
#include <algorithm>
#include <cmath>

#include "mm_ctx.h"

namespace mm {
namespace {

// Shared-memory histograms: up to 96 KB per CTA (8 warp copies of 512 bins per map, 32 KB);
// 200 KB of an SM's shared memory shared between the CTAs of a launch.
constexpr size_t kHistSmemMax = 96 * 1024;
constexpr size_t kSmemPerSm = 200 * 1024;

struct StatSums {
    double sum_sq;                 // sum of (Delta m_a - Delta m_b)^2 over pixels counted in both maps
    unsigned long long n_both;
    unsigned long long zero_a, zero_b;
    unsigned long long sum_a, sum_b;
    unsigned int max_count;
    int pad;
    long long ks_num;              // max_k |c_a(k) n_b - c_b(k) n_a|
};

// Pass 1 over both maps: sums, empty pixels and the largest count (no logarithms).
__global__ void k_scan_stats(const unsigned *a, const unsigned *b, long long n, StatSums *out)
{
    unsigned long long za = 0, zb = 0, sa = 0, sb = 0;
    unsigned mx = 0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const unsigned na = a[k], nb = b[k];
        sa += na;
        sb += nb;
        mx = max(mx, max(na, nb));
        za += na == 0u;
        zb += nb == 0u;
    }
    for (int o = 16; o > 0; o >>= 1) {
        za += __shfl_down_sync(0xffffffffu, za, o);
        zb += __shfl_down_sync(0xffffffffu, zb, o);
        sa += __shfl_down_sync(0xffffffffu, sa, o);
        sb += __shfl_down_sync(0xffffffffu, sb, o);
        mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out->zero_a, za);
        atomicAdd(&out->zero_b, zb);
        atomicAdd(&out->sum_a, sa);
        atomicAdd(&out->sum_b, sb);
        atomicMax(&out->max_count, mx);
    }
}

// Per count k >= 1 that a pixel can hold, Delta m up to the factor -2.5 of each map,
// log10(k) - log10(N_rays), as a float-float pair (hi, lo) of its FP64 value: pass 2
// then forms the per-pixel differences in FP32 arithmetic (the FP64 pipe runs at 1/64 of
// the FP32 rate). ta[0], tb[0] unused.
__global__ void k_log_table(long long nbins, double log10_ra, double log10_rb, float2 *ta, float2 *tb)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nbins; k += (long long)gridDim.x * blockDim.x) {
        const double l = k ? log10((double)k) : 0.0, va = l - log10_ra, vb = l - log10_rb;
        const float ah = __double2float_rn(va), bh = __double2float_rn(vb);
        ta[k] = make_float2(ah, __double2float_rn(va - (double)ah));
        tb[k] = make_float2(bh, __double2float_rn(vb - (double)bh));
    }
}

// Float-float helpers (error-free transformations: Knuth's TwoSum, FMA-based TwoProd).
__device__ __forceinline__ void ff_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (sh, sl) += (ph, pl), renormalised.
__device__ __forceinline__ void ff_accumulate(float &sh, float &sl, float ph, float pl)
{
    float s, e;
    ff_two_sum(sh, ph, s, e);
    e = __fadd_rn(e, __fadd_rn(sl, pl));
    sh = __fadd_rn(s, e);
    sl = __fsub_rn(e, __fsub_rn(sh, s));
}

// Add 1 to h[key] for every lane holding key (skipped: kNoKey); lanes with equal keys
// are merged first, so a warp issues one atomic per distinct key.
constexpr unsigned kNoKey = 0xffffffffu;

__device__ __forceinline__ void hist_add(unsigned *h, unsigned key, unsigned lane)
{
    const unsigned same = __match_any_sync(0xffffffffu, key);
    if (key != kNoKey && lane == (unsigned)(__ffs(same) - 1)) atomicAdd(h + key, (unsigned)__popc(same));
}

// Pass 2 over both maps: the RMS of Delta m_a - Delta m_b over pixels counted in both,
//   Delta m_a - Delta m_b = -2.5 [(log10 N_a - log10 N_rays_a) - (log10 N_b - log10 N_rays_b)]
//                         = -2.5 (ta[N_a] - tb[N_b]),
// the difference and its square in float-float (about 1e-14 relative), summed per thread in
// float-float and then in FP64; and the two count histograms (bins 0 .. nbins - 1,
// nbins = largest count + 1) added to ha / hb. Each warp keeps its own copy of the bins below
// wb = min(nbins, kWarpBins) in shared memory and adds to it with plain shared-memory atomics:
// only the lanes of one warp can collide on a bin, so no merging of equal keys is needed for the
// common small counts. The rare larger counts go to the global histograms, merged per warp.
// A thread takes four consecutive pixels of each map per step (16-byte loads; the counts come
// from the arena, 256-byte aligned), so that several loads and table lookups are in flight; the
// last n % 4 pixels go to the first threads of block 0. (Two such groups per step were timed and
// kept out: 205 against 192 us on two 8192^2 maps.)
constexpr int kWarpBins = 512;

__device__ __forceinline__ void rms_pixel(unsigned na, unsigned nb, const float2 *ta, const float2 *tb, float &qh,
                                          float &ql, unsigned long long &both)
{
    if (na && nb) {
        // d = ta[na] - tb[nb] in float-float, then d^2
        const float2 x = ta[na], y = tb[nb];
        float dh, dl;
        ff_two_sum(x.x, -y.x, dh, dl);
        dl = __fadd_rn(dl, __fsub_rn(x.y, y.y));
        const float d = __fadd_rn(dh, dl), de = __fsub_rn(dl, __fsub_rn(d, dh));
        const float ph = __fmul_rn(d, d);
        const float pl = __fmaf_rn(d, d, -ph) + 2.f * d * de;
        ff_accumulate(qh, ql, ph, pl);
        both += 1;
    }
}

// Count keys na, nb of one lane (in: the lane holds a pixel) into the warp's bins, or, for
// counts of wb or more, into the global histograms.
__device__ __forceinline__ void hist_pixel(bool in, unsigned na, unsigned nb, unsigned *sa, unsigned *sb,
                                           unsigned *ha, unsigned *hb, long long wb, unsigned lane)
{
    if (in && na < (unsigned)wb) atomicAdd(sa + na, 1u);
    if (in && nb < (unsigned)wb) atomicAdd(sb + nb, 1u);
    const bool big_a = in && na >= (unsigned)wb, big_b = in && nb >= (unsigned)wb;
    if (__any_sync(0xffffffffu, big_a)) hist_add(ha, big_a ? na : kNoKey, lane);
    if (__any_sync(0xffffffffu, big_b)) hist_add(hb, big_b ? nb : kNoKey, lane);
}

__global__ void __launch_bounds__(256) k_rms_hist(const unsigned *a, const unsigned *b, long long n, const float2 *ta,
                                                  const float2 *tb, long long nbins, unsigned *ha, unsigned *hb,
                                                  StatSums *out)
{
    extern __shared__ unsigned sh[];                          // [8 warps][2 maps][wb]
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long wb = min(nbins, (long long)kWarpBins);
    unsigned *const sa = sh + warp * 2 * wb, *const sb = sa + wb;
    for (long long k = threadIdx.x; k < 16 * wb; k += blockDim.x) sh[k] = 0u;
    __syncthreads();
    float qh = 0.f, ql = 0.f;                                 // float-float sum of (Delta m_a - Delta m_b)^2 / 6.25
    unsigned long long both = 0;
    const uint4 *a4 = reinterpret_cast<const uint4 *>(a), *b4 = reinterpret_cast<const uint4 *>(b);
    const long long n4 = n / 4;
    // warp-uniform trip count: the lanes of a warp take consecutive groups, those past n4 hold no key
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long w0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31u); w0 < n4; w0 += stride) {
        const long long k = w0 + lane;
        const bool in = k < n4;
        const uint4 va = in ? a4[k] : make_uint4(0u, 0u, 0u, 0u), vb = in ? b4[k] : make_uint4(0u, 0u, 0u, 0u);
        rms_pixel(va.x, vb.x, ta, tb, qh, ql, both);
        rms_pixel(va.y, vb.y, ta, tb, qh, ql, both);
        rms_pixel(va.z, vb.z, ta, tb, qh, ql, both);
        rms_pixel(va.w, vb.w, ta, tb, qh, ql, both);
        hist_pixel(in, va.x, vb.x, sa, sb, ha, hb, wb, lane);
        hist_pixel(in, va.y, vb.y, sa, sb, ha, hb, wb, lane);
        hist_pixel(in, va.z, vb.z, sa, sb, ha, hb, wb, lane);
        hist_pixel(in, va.w, vb.w, sa, sb, ha, hb, wb, lane);
    }
    if (blockIdx.x == 0 && warp == 0) {                        // the last n % 4 pixels
        const long long k = 4 * n4 + lane;
        const bool in = k < n;
        const unsigned na = in ? a[k] : 0u, nb = in ? b[k] : 0u;
        rms_pixel(na, nb, ta, tb, qh, ql, both);
        hist_pixel(in, na, nb, sa, sb, ha, hb, wb, lane);
    }
    double sq = 6.25 * ((double)qh + (double)ql);              // Delta m differences carry the factor -2.5
    for (int o = 16; o > 0; o >>= 1) {
        sq += __shfl_down_sync(0xffffffffu, sq, o);
        both += __shfl_down_sync(0xffffffffu, both, o);
    }
    if (lane == 0) {
        atomicAdd(&out->sum_sq, sq);
        atomicAdd(&out->n_both, both);
    }
    __syncthreads();
    for (long long k = threadIdx.x; k < 2 * wb; k += blockDim.x) {   // the 8 warp copies of each bin
        unsigned v = 0;
        for (int q = 0; q < 8; ++q) v += sh[q * 2 * wb + k];
        if (v) atomicAdd(k < wb ? ha + k : hb + (k - wb), v);
    }
}

// One CTA of 1024 threads: inclusive prefix sums ca[k], cb[k] of the two count
// histograms (so P(N >= k) = (n - c[k-1]) / n).
__global__ void __launch_bounds__(1024) k_scan(const unsigned *ha, const unsigned *hb, long long nbins, long long *ca,
                                               long long *cb)
{
    __shared__ long long sa[1024], sb[1024];
    const int t = threadIdx.x;
    const long long per = (nbins + 1023) / 1024;
    const long long lo = min(nbins, t * per), hi = min(nbins, lo + per);
    long long ta = 0, tb = 0;
    for (long long k = lo; k < hi; ++k) {
        ta += ha[k];
        tb += hb[k];
    }
    sa[t] = ta;
    sb[t] = tb;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {           // inclusive scan of the per-thread totals
        const long long va = (t >= o) ? sa[t - o] : 0, vb = (t >= o) ? sb[t - o] : 0;
        __syncthreads();
        sa[t] += va;
        sb[t] += vb;
        __syncthreads();
    }
    ta = (t > 0) ? sa[t - 1] : 0;
    tb = (t > 0) ? sb[t - 1] : 0;
    for (long long k = lo; k < hi; ++k) {
        ta += ha[k];
        tb += hb[k];
        ca[k] = ta;
        cb[k] = tb;
    }
}

// Number of samples of a map with mu = N / nr >= m: n - c[kmin - 1], kmin the smallest
// count with kmin / nr >= m (divisions correctly rounded, as in the oracle's Delta m).
__device__ __forceinline__ long long survivors(const long long *c, long long nbins, long long n, double nr, double m)
{
    long long k = (long long)ceil(m * nr);
    if (k < 0) k = 0;
    while (k > 0 && __ddiv_rn((double)(k - 1), nr) >= m) --k;
    while (k < nbins && __ddiv_rn((double)k, nr) < m) ++k;
    if (k >= nbins) return 0;
    return n - (k > 0 ? c[k - 1] : 0);
}

// D numerator: max over every value mu = k / nr present in either map of
// |S_a(mu) n_b - S_b(mu) n_a|, S the survivor counts; the K-S supremum over Delta m
// thresholds is attained at these points (Delta m is decreasing in mu).
__global__ void k_ks_eval(const unsigned *ha, const unsigned *hb, const long long *ca, const long long *cb,
                          long long nbins, long long na, long long nb, double ra, double rb, StatSums *out)
{
    long long best = 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 2 * nbins;
         q += (long long)gridDim.x * blockDim.x) {
        const bool from_a = q < nbins;
        const long long k = from_a ? q : q - nbins;
        if ((from_a ? ha[k] : hb[k]) == 0u) continue;
        const double m = __ddiv_rn((double)k, from_a ? ra : rb);
        const long long sa = survivors(ca, nbins, na, ra, m), sb = survivors(cb, nbins, nb, rb, m);
        const long long d = sa * nb - sb * na;
        best = max(best, d < 0 ? -d : d);
    }
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_down_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long *)&out->ks_num, (unsigned long long)best);
}

// Kolmogorov distribution survival function Q(l) = 2 sum (-1)^(j-1) exp(-2 j^2 l^2).
double kolmogorov_q(double l)
{
    if (l < 0.2) return 1.0;
    double s = 0.0, sign = 1.0;
    for (int j = 1; j <= 200; ++j) {
        const double term = std::exp(-2.0 * j * j * l * l);
        s += sign * term;
        if (term < 1e-17) break;
        sign = -sign;
    }
    return std::min(1.0, std::max(0.0, 2.0 * s));
}

}  // namespace
}  // namespace mm

using namespace mm;

extern "C" int mm_map_compare(mm_ctx *ctx, mm_map a, mm_map b, mm_compare *out)
{
    if (!ctx || !out) return fail(MM_EINVAL, "null argument");
    std::shared_ptr<MapObj> A, B;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto ia = ctx->maps.find(a), ib = ctx->maps.find(b);
        if (ia == ctx->maps.end() || ib == ctx->maps.end()) return fail(MM_ENOTFOUND, "unknown map");
        A = ia->second;
        B = ib->second;
    }
    if (A->p.npix_side != B->p.npix_side) return fail(MM_EINVAL, "maps of different N_side");
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    cudaError_t e;
    if ((e = cudaStreamWaitEvent(s, A->done, 0)) != cudaSuccess || (e = cudaStreamWaitEvent(s, B->done, 0)) != cudaSuccess)
        return cuda_fail(e, "wait for maps");
    const long long n = (long long)A->p.npix_side * A->p.npix_side;
    struct Tmp {
        DeviceArena *ar;
        std::vector<void *> v;
        ~Tmp() { for (void *p : v) ar->free(p); }
    } tmp{&ctx->arena, {}};
    StatSums *d_sum = nullptr;
    int rc = ctx->arena.alloc(sizeof(StatSums), (void **)&d_sum);
    if (rc) return rc;
    tmp.v.push_back(d_sum);
    if ((e = cudaMemsetAsync(d_sum, 0, sizeof(StatSums), s)) != cudaSuccess) return cuda_fail(e, "memset");
    const int grid = std::max(1, std::min(4 * ctx->sms, (int)((n + 255) / 256)));
    k_scan_stats<<<grid, 256, 0, s>>>(A->counts, B->counts, n, d_sum);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "k_scan_stats");
    StatSums h{};
    if ((e = cudaMemcpyAsync(&h, d_sum, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "stats readback");
    // log10 table over the counts, histograms of the counts over 0..max with the RMS pass,
    // then their prefix sums and the exact K-S numerator
    const long long nbins = (long long)h.max_count + 1;
    unsigned *hist = nullptr;
    long long *cum = nullptr;
    float2 *tab = nullptr;                                     // [2 nbins]: map a, then map b
    if ((rc = ctx->arena.alloc((size_t)(2 * nbins) * sizeof(unsigned), (void **)&hist))) return rc;
    tmp.v.push_back(hist);
    if ((rc = ctx->arena.alloc((size_t)(2 * nbins) * sizeof(long long), (void **)&cum))) return rc;
    tmp.v.push_back(cum);
    if ((rc = ctx->arena.alloc((size_t)(2 * nbins) * sizeof(float2), (void **)&tab))) return rc;
    tmp.v.push_back(tab);
    if ((e = cudaMemsetAsync(hist, 0, (size_t)(2 * nbins) * sizeof(unsigned), s)) != cudaSuccess) return cuda_fail(e, "memset");
    const double lra = std::log10(A->p.nrays_per_pix), lrb = std::log10(B->p.nrays_per_pix);
    k_log_table<<<std::max(1, std::min(ctx->sms, (int)((nbins + 255) / 256))), 256, 0, s>>>(nbins, lra, lrb, tab,
                                                                                           tab + nbins);
    // histograms: per warp in shared memory (the bins below kWarpBins), so that the common small
    // counts need no merging of equal keys; the few larger counts go to the global histograms
    const size_t smem = (size_t)16 * (size_t)std::min<long long>(nbins, kWarpBins) * sizeof(unsigned);
    if ((e = cudaFuncSetAttribute(k_rms_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kHistSmemMax)) != cudaSuccess)
        return cuda_fail(e, "k_rms_hist shared memory");
    {
        const int per_sm = std::max(1, std::min(6, (int)(kSmemPerSm / std::max<size_t>(smem, 1))));
        k_rms_hist<<<std::max(1, std::min(per_sm * ctx->sms, (int)((n + 255) / 256))), 256, smem, s>>>(
            A->counts, B->counts, n, tab, tab + nbins, nbins, hist, hist + nbins, d_sum);
    }
    k_scan<<<1, 1024, 0, s>>>(hist, hist + nbins, nbins, cum, cum + nbins);
    const int egrid = std::max(1, std::min(4 * ctx->sms, (int)((2 * nbins + 255) / 256)));
    k_ks_eval<<<egrid, 256, 0, s>>>(hist, hist + nbins, cum, cum + nbins, nbins, n, n, A->p.nrays_per_pix,
                                    B->p.nrays_per_pix, d_sum);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "k_rms_hist/k_scan/k_ks_eval");
    if ((e = cudaMemcpyAsync(&h, d_sum, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "stats readback");
    out->n_rms = (int64_t)h.n_both;
    out->rms_dm = h.n_both ? std::sqrt(h.sum_sq / (double)h.n_both) : 0.0;
    out->zero_a = (int64_t)h.zero_a;
    out->zero_b = (int64_t)h.zero_b;
    out->ks_d = (double)h.ks_num / ((double)n * (double)n);
    const double ne = (double)n * (double)n / (2.0 * (double)n), sq = std::sqrt(ne);
    out->ks_p = kolmogorov_q((sq + 0.12 + 0.11 / sq) * out->ks_d);
    out->mean_mu_a = (double)h.sum_a / ((double)n * A->p.nrays_per_pix);
    out->mean_mu_b = (double)h.sum_b / ((double)n * B->p.nrays_per_pix);
    return MM_OK;
}

// ---- normalised maps (Sect. 2, the estimator; Eq. deltam) ------------------------

namespace mm {
namespace {

// Per pixel mu = N / N_rays, or Delta m = -2.5 log10(max(N, 1) / N_rays) (an empty pixel
// is clamped to one ray, which bounds its Delta m), in FP32 from the uint32 counts; the
// number of empty pixels goes to *n_empty. Four pixels per thread and step (16-byte loads
// and stores; both buffers come from the arena, 256-byte aligned), the last n % 4 pixels
// by the first threads of block 0.
__global__ void __launch_bounds__(256) k_map_normalise(const unsigned *c, long long n, int kind, float inv_nrays,
                                                       float log10_nrays, float *out, unsigned long long *n_empty)
{
    auto one = [&](unsigned v) {
        return kind == MM_MAP_DELTA_M ? -2.5f * (log10f((float)max(v, 1u)) - log10_nrays) : (float)v * inv_nrays;
    };
    unsigned long long z = 0;
    const long long n4 = n / 4;
    const uint4 *c4 = reinterpret_cast<const uint4 *>(c);
    float4 *o4 = reinterpret_cast<float4 *>(out);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n4; k += (long long)gridDim.x * blockDim.x) {
        const uint4 v = c4[k];
        o4[k] = make_float4(one(v.x), one(v.y), one(v.z), one(v.w));
        z += (v.x == 0u) + (v.y == 0u) + (v.z == 0u) + (v.w == 0u);
    }
    if (blockIdx.x == 0 && threadIdx.x < n - 4 * n4) {
        const long long k = 4 * n4 + threadIdx.x;
        out[k] = one(c[k]);
        z += c[k] == 0u;
    }
    z = __reduce_add_sync(0xffffffffu, (unsigned)z);
    if ((threadIdx.x & 31) == 0 && z) atomicAdd(n_empty, z);
}

}  // namespace
}  // namespace mm

extern "C" int mm_map_fetch_mu(mm_ctx *ctx, mm_map map, int32_t kind, float *host_out, size_t n_elems,
                               int64_t *n_empty)
{
    if (!ctx) return fail(MM_EINVAL, "null context");
    if (kind != MM_MAP_MU && kind != MM_MAP_DELTA_M) return fail(MM_EINVAL, "kind must be MM_MAP_MU or MM_MAP_DELTA_M");
    std::shared_ptr<MapObj> M;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->maps.find(map);
        if (it == ctx->maps.end()) return fail(MM_ENOTFOUND, "unknown map");
        M = it->second;
    }
    const long long n = (long long)M->p.npix_side * M->p.npix_side;
    if (!host_out || n_elems != (size_t)n) return fail(MM_EINVAL, "host buffer must hold N_side^2 floats");
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    cudaError_t e;
    if ((e = cudaStreamWaitEvent(s, M->done, 0)) != cudaSuccess) return cuda_fail(e, "wait for map");
    float *buf = nullptr;
    int rc = ctx->arena.alloc((size_t)n * sizeof(float) + 256, (void **)&buf);
    if (rc) return rc;
    unsigned long long *d_empty = reinterpret_cast<unsigned long long *>(buf + n + (4 - n % 4) % 4);
    unsigned long long h_empty = 0;
    const double nr = M->p.nrays_per_pix;
    const int grid = std::max(1, std::min(4 * ctx->sms, (int)((n / 4 + 255) / 256)));
    if ((e = cudaMemsetAsync(d_empty, 0, sizeof(unsigned long long), s)) == cudaSuccess) {
        k_map_normalise<<<grid, 256, 0, s>>>(M->counts, n, kind, (float)(1.0 / nr), (float)std::log10(nr), buf,
                                             d_empty);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, buf, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_empty, d_empty, sizeof(h_empty), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    ctx->arena.free(buf);
    if (e != cudaSuccess) return cuda_fail(e, "normalised map");
    if (n_empty) *n_empty = (int64_t)h_empty;
    return MM_OK;
}
