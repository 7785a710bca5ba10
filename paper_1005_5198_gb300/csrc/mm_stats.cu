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

#include "mm_async.cuh"
#include "mm_ctx.h"

namespace mm {
namespace {

// The comparison reads both maps once (k_compare), streaming them through shared memory in chunks
// of kCmpChunk bytes per map: a producer warp keeps kCmpStages chunks in flight with bulk copies,
// and 4 consumer warps read each chunk's pixels with 16-byte loads (two groups of 4 pixels per lane
// and map), releasing its stage per warp. Histograms: the bins below kWarpBins in shared memory, one
// copy per pair of consumer warps (2 copies x 2 maps x 1024 bins, 16 KB); 48 KB of shared memory per
// CTA, 4 CTAs per SM.
constexpr int kCmpConsumers = 4;
constexpr int kCmpThreads = 32 * (kCmpConsumers + 1);
constexpr int kCmpStages = 4;
constexpr int kCmpChunk = 4096;
constexpr int kWarpBins = 1024;
constexpr int kBinCopies = kCmpConsumers / 2;
constexpr size_t kCmpSmem = (size_t)kCmpStages * 2 * kCmpChunk + 128 + (size_t)kBinCopies * 2 * kWarpBins * 4;

struct StatSums {
    double sum_sq;                 // sum of (Delta m_a - Delta m_b)^2 over pixels counted in both maps
    unsigned long long n_both;
    unsigned long long zero_a, zero_b;
    unsigned long long sum_a, sum_b;
    unsigned int max_count;        // largest count of nbins or more (0: none)
    unsigned int fault;            // a copy into shared memory did not complete in time
    long long ks_num;              // max_k |c_a(k) n_b - c_b(k) n_a|
    unsigned long long over_a, over_b;   // pixels with counts of nbins or more (sent to the lists)
};

// Delta m up to the factor -2.5 of a count k >= 1 of a map with N_rays = 10^lr,
// log10(k) - lr, as a float-float pair (hi, lo) of its FP64 value: the RMS then forms the
// per-pixel differences in FP32 arithmetic (the FP64 pipe runs at 1/64 of the FP32 rate).
__device__ __forceinline__ float2 log_pair(unsigned k, double lr)
{
    const double v = (k ? log10((double)k) : 0.0) - lr;
    const float hi = __double2float_rn(v);
    return make_float2(hi, __double2float_rn(v - (double)hi));
}

// The pairs of every count below nbins, for both maps (ta[0], tb[0] unused); larger counts are
// converted where they occur, by the same function, so that every pixel sees the same value.
__global__ void k_log_table(long long nbins, double log10_ra, double log10_rb, float2 *ta, float2 *tb)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nbins; k += (long long)gridDim.x * blockDim.x) {
        ta[k] = log_pair((unsigned)k, log10_ra);
        tb[k] = log_pair((unsigned)k, log10_rb);
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

// Per-thread running totals of k_compare.
struct CmpAcc {
    float qh = 0.f, ql = 0.f;                  // float-float sum of (Delta m_a - Delta m_b)^2 / 6.25
    unsigned both = 0;                         // pixels counted in both maps
    unsigned big_max = 0;                      // largest listed count
};

// What k_compare computes and where it sends each count.
struct CmpArgs {
    const float2 *ta, *tb;                     // log pairs of the counts below nbins
    double lra, lrb;                           // log10 N_rays of each map
    long long nbins;                           // bins of ha, hb
    unsigned *ha, *hb;                         // histograms of the counts below nbins
    unsigned *la, *lb;                         // counts of nbins or more, listed (room for cap each)
    unsigned long long cap;
    int hist_only;                             // 1: histograms alone (every count is below nbins)
    int no_copy;                               // test hook: the producer issues no copies
};

// The RMS term of one pixel:
//   Delta m_a - Delta m_b = -2.5 [(log10 N_a - log10 N_rays_a) - (log10 N_b - log10 N_rays_b)]
//                         = -2.5 (pair_a(N_a) - pair_b(N_b)),
// the difference and its square in float-float (about 1e-14 relative), over pixels counted in both.
// The square of pair_a - pair_b in float-float, added to the running sum (zero for a pixel empty in
// either map: every pixel runs the arithmetic, so that a warp does not diverge).
__device__ __forceinline__ void rms_add(float2 x, float2 y, bool use, CmpAcc &acc)
{
    float dh, dl;
    ff_two_sum(x.x, -y.x, dh, dl);
    dl = __fadd_rn(dl, __fsub_rn(x.y, y.y));
    const float d = __fadd_rn(dh, dl), de = __fsub_rn(dl, __fsub_rn(d, dh));
    const float ph = __fmul_rn(d, d);
    const float pl = __fmaf_rn(d, d, -ph) + 2.f * d * de;
    ff_accumulate(acc.qh, acc.ql, use ? ph : 0.f, use ? pl : 0.f);
    acc.both += use;
}

__device__ __forceinline__ void rms_pixel(unsigned na, unsigned nb, const CmpArgs &g, CmpAcc &acc)
{
    const float2 x = na < (unsigned long long)g.nbins ? __ldg(g.ta + na) : log_pair(na, g.lra);
    const float2 y = nb < (unsigned long long)g.nbins ? __ldg(g.tb + nb) : log_pair(nb, g.lrb);
    rms_add(x, y, na && nb, acc);
}

// The same for counts known to be below nbins.
__device__ __forceinline__ void rms_pixel_small(unsigned na, unsigned nb, const CmpArgs &g, CmpAcc &acc)
{
    rms_add(__ldg(g.ta + na), __ldg(g.tb + nb), na && nb, acc);
}

// Count the key of one lane (in: the lane holds a pixel) into the warp's shared bins (keys below
// kWarpBins), the global histogram (below nbins, merged per warp) or the list of large counts.
__device__ __forceinline__ void hist_key(bool in, unsigned key, unsigned *sbins, unsigned *h, unsigned *list,
                                         unsigned long long *n_list, unsigned long long cap, long long nbins,
                                         unsigned &big_max, unsigned lane)
{
    if (in && key < (unsigned)kWarpBins) atomicAdd(sbins + key, 1u);
    const bool mid = in && key >= (unsigned)kWarpBins && key < (unsigned long long)nbins;
    if (__any_sync(0xffffffffu, mid)) hist_add(h, mid ? key : kNoKey, lane);
    const bool big = in && key >= (unsigned long long)nbins;
    const unsigned bigm = __ballot_sync(0xffffffffu, big);
    if (bigm) {
        unsigned long long base = 0;
        if (lane == (unsigned)(__ffs(bigm) - 1)) base = atomicAdd(n_list, (unsigned long long)__popc(bigm));
        base = __shfl_sync(0xffffffffu, base, __ffs(bigm) - 1);
        const unsigned long long slot = base + __popc(bigm & ((1u << lane) - 1u));
        if (big && slot < cap) list[slot] = key;
        if (big) big_max = max(big_max, key);
    }
}

// Four pixels of each map held by every lane of a warp (in: the lane holds pixels). When every
// count of the warp's 256 is below kWarpBins (the usual case; kWarpBins <= nbins) the RMS reads the
// tables directly and the keys go straight to the shared bins; otherwise the keys below kWarpBins
// still do, and the larger ones take hist_key's way, one key position at a time.
__device__ __forceinline__ void cmp_quad(bool in, uint4 x, uint4 y, const CmpArgs &g, CmpAcc &acc, unsigned *sa,
                                         unsigned *sb, StatSums *out, unsigned lane)
{
    const unsigned m = max(max(max(x.x, x.y), max(x.z, x.w)), max(max(y.x, y.y), max(y.z, y.w)));
    const unsigned ka[4] = {x.x, x.y, x.z, x.w}, kb[4] = {y.x, y.y, y.z, y.w};
    if (__all_sync(0xffffffffu, m < (unsigned)kWarpBins)) {
        if (!g.hist_only) {
#pragma unroll
            for (int u = 0; u < 4; ++u) rms_pixel_small(ka[u], kb[u], g, acc);
        }
        if (in) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                atomicAdd(sa + ka[u], 1u);
                atomicAdd(sb + kb[u], 1u);
            }
        }
        return;
    }
    if (!g.hist_only) {
#pragma unroll
        for (int u = 0; u < 4; ++u) rms_pixel(ka[u], kb[u], g, acc);
    }
    if (in) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (ka[u] < (unsigned)kWarpBins) atomicAdd(sa + ka[u], 1u);
            if (kb[u] < (unsigned)kWarpBins) atomicAdd(sb + kb[u], 1u);
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {                          // only keys of kWarpBins or more are left
        hist_key(in && ka[u] >= (unsigned)kWarpBins, ka[u], sa, g.ha, g.la, &out->over_a, g.cap, g.nbins, acc.big_max,
                 lane);
        hist_key(in && kb[u] >= (unsigned)kWarpBins, kb[u], sb, g.hb, g.lb, &out->over_b, g.cap, g.nbins, acc.big_max,
                 lane);
    }
}

// One pass over both maps: the RMS of Delta m_a - Delta m_b and the count histograms below nbins,
// with the larger counts listed (their number per map and the largest go to out). A CTA takes
// chunks blockIdx.x, blockIdx.x + gridDim.x, ... of kCmpChunk bytes of each map (the first
// 4 floor(n / 4) pixels; the last n % 4 go to consumer warp 0 of block 0 with plain loads).
// Lane 0 of the producer warp (warp 8) fills stage i % kCmpStages with chunk i once the 8 consumer
// warps have released it (empty barrier), and the copies complete on the stage's full barrier.
// A wait that runs out of time sets out->fault and ends that warp's loop; the producer then waits
// (again with the limit) for the copies it issued, so that none lands after the CTA has left.
__global__ void __launch_bounds__(kCmpThreads) k_compare(const unsigned *a, const unsigned *b, long long n, CmpArgs g,
                                                          StatSums *out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint4 *const stage = reinterpret_cast<uint4 *>(smem);                     // [stage][map][chunk / 16]
    uint64_t *const full = reinterpret_cast<uint64_t *>(smem + (size_t)kCmpStages * 2 * kCmpChunk);
    uint64_t *const empty = full + kCmpStages;
    unsigned *const bins = reinterpret_cast<unsigned *>(smem + (size_t)kCmpStages * 2 * kCmpChunk + 128);
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < kBinCopies * 2 * kWarpBins; k += kCmpThreads) bins[k] = 0u;
    const long long bytes = (n / 4) * 16;
    const long long chunks = (bytes + kCmpChunk - 1) / kCmpChunk;
    const long long mine = chunks > blockIdx.x ? (chunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto chunk_bytes = [&](long long i) {
        const long long off = (blockIdx.x + i * gridDim.x) * (long long)kCmpChunk;
        return (unsigned)min((long long)kCmpChunk, bytes - off);
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s < kCmpStages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, kCmpConsumers);
        }
        mbar_fence_init();
    }
    __syncthreads();
    CmpAcc acc;
    if (warp == kCmpConsumers) {                                             // producer
        if (lane == 0) {
            long long issued = 0;
            for (long long i = 0; i < (g.no_copy ? 0 : mine); ++i) {
                const int s = (int)(i % kCmpStages);
                if (i >= kCmpStages && !mbar_wait(empty + s, (unsigned)((i / kCmpStages - 1) & 1))) {
                    atomicExch(&out->fault, 1u);
                    break;
                }
                const long long off = (blockIdx.x + i * gridDim.x) * (long long)kCmpChunk;
                const unsigned nb = chunk_bytes(i);
                mbar_arrive_expect(full + s, 2 * nb);
                bulk_load(stage + (size_t)s * 2 * (kCmpChunk / 16), reinterpret_cast<const unsigned char *>(a) + off,
                          nb, full + s);
                bulk_load(stage + ((size_t)s * 2 + 1) * (kCmpChunk / 16),
                          reinterpret_cast<const unsigned char *>(b) + off, nb, full + s);
                issued = i + 1;
            }
            // every issued copy has landed before the CTA leaves (normally the consumers saw them all)
            for (long long j = max(0LL, issued - kCmpStages); j < issued; ++j)
                if (!mbar_wait(full + (int)(j % kCmpStages), (unsigned)((j / kCmpStages) & 1)))
                    atomicExch(&out->fault, 1u);
        }
    } else {                                                                 // consumers
        unsigned *const sa = bins + (warp >> 1) * 2 * kWarpBins, *const sb = sa + kWarpBins;
        for (long long i = 0; i < mine; ++i) {
            const int s = (int)(i % kCmpStages);
            // every lane waits (and so sees the copies); the warp goes on only if all of them saw it
            if (!__all_sync(0xffffffffu, mbar_wait(full + s, (unsigned)((i / kCmpStages) & 1)))) {
                if (lane == 0) atomicExch(&out->fault, 1u);
                break;
            }
            const uint4 *const va = stage + (size_t)s * 2 * (kCmpChunk / 16), *const vb = va + kCmpChunk / 16;
            if (i + 1 < mine || bytes % kCmpChunk == 0) {                    // a whole chunk
#pragma unroll
                for (int q0 = warp * 32; q0 < kCmpChunk / 16; q0 += 32 * kCmpConsumers)
                    cmp_quad(true, va[q0 + lane], vb[q0 + lane], g, acc, sa, sb, out, lane);
            } else {                                                         // the last, shorter chunk
                const int quads = (int)(chunk_bytes(i) / 16);
                for (int q0 = warp * 32; q0 < quads; q0 += 32 * kCmpConsumers) {  // warp-uniform trip count
                    const int q = q0 + (int)lane;
                    const bool in = q < quads;
                    cmp_quad(in, in ? va[q] : make_uint4(0u, 0u, 0u, 0u), in ? vb[q] : make_uint4(0u, 0u, 0u, 0u), g,
                             acc, sa, sb, out, lane);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty + s);                           // this warp is done with stage s
        }
        if (blockIdx.x == 0 && warp == 0) {                                  // the last n % 4 pixels, one each
            const long long k = 4 * (n / 4) + lane;
            const bool in = k < n;
            const unsigned ka = in ? a[k] : 0u, kb = in ? b[k] : 0u;
            if (!g.hist_only) rms_pixel(ka, kb, g, acc);
            hist_key(in, ka, sa, g.ha, g.la, &out->over_a, g.cap, g.nbins, acc.big_max, lane);
            hist_key(in, kb, sb, g.hb, g.lb, &out->over_b, g.cap, g.nbins, acc.big_max, lane);
        }
        double sq = 6.25 * ((double)acc.qh + (double)acc.ql);                // Delta m differences carry -2.5
        unsigned long long both = acc.both;
        for (int o = 16; o > 0; o >>= 1) {
            sq += __shfl_down_sync(0xffffffffu, sq, o);
            both += __shfl_down_sync(0xffffffffu, both, o);
            acc.big_max = max(acc.big_max, __shfl_down_sync(0xffffffffu, acc.big_max, o));
        }
        if (lane == 0) {
            if (!g.hist_only) {
                atomicAdd(&out->sum_sq, sq);
                atomicAdd(&out->n_both, both);
            }
            if (acc.big_max) atomicMax(&out->max_count, acc.big_max);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * kWarpBins; k += kCmpThreads) {         // the copies of each bin
        unsigned v = 0;
        for (int q = 0; q < kBinCopies; ++q) v += bins[q * 2 * kWarpBins + k];
        if (v) atomicAdd(k < kWarpBins ? g.ha + k : g.hb + (k - kWarpBins), v);
    }
}

// The listed large counts of one map added to its histogram (bins up to the largest count).
__global__ void k_list_hist(const unsigned *list, unsigned long long m, unsigned *h)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)m; k += (long long)gridDim.x * blockDim.x)
        atomicAdd(h + list[k], 1u);
}

// One CTA of 1024 threads: inclusive prefix sums ca[k], cb[k] of the two count
// histograms (so P(N >= k) = (n - c[k-1]) / n), and from the histograms the empty pixels
// (bin 0) and the total count sum_k k h[k] of each map, written to out. Thread t takes a run of
// consecutive bins; the runs' totals are scanned with warp shuffles (within a warp, then over the
// 32 warp totals).
__device__ __forceinline__ long long warp_incl_scan(long long v, unsigned lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (unsigned)o) v += u;
    }
    return v;
}

__global__ void __launch_bounds__(1024) k_scan(const unsigned *ha, const unsigned *hb, long long nbins, long long *ca,
                                               long long *cb, StatSums *out)
{
    __shared__ long long wa[32], wb[32];
    __shared__ unsigned long long wsum[2][32];
    const int t = threadIdx.x;
    const unsigned lane = t & 31, warp = t >> 5;
    const long long per = (nbins + 1023) / 1024;
    const long long lo = min(nbins, t * per), hi = min(nbins, lo + per);
    long long ta = 0, tb = 0;
    unsigned long long ma = 0, mb = 0;             // sum of k h[k] over this thread's bins
    for (long long k = lo; k < hi; ++k) {
        ta += ha[k];
        tb += hb[k];
        ma += (unsigned long long)k * ha[k];
        mb += (unsigned long long)k * hb[k];
    }
    for (int o = 16; o > 0; o >>= 1) {
        ma += __shfl_down_sync(0xffffffffu, ma, o);
        mb += __shfl_down_sync(0xffffffffu, mb, o);
    }
    const long long ia = warp_incl_scan(ta, lane), ib = warp_incl_scan(tb, lane);
    if (lane == 31) {
        wa[warp] = ia;
        wb[warp] = ib;
    }
    if (lane == 0) {
        wsum[0][warp] = ma;
        wsum[1][warp] = mb;
    }
    __syncthreads();
    if (warp == 0) {                               // exclusive scan of the warp totals
        const long long xa = warp_incl_scan(wa[lane], lane), xb = warp_incl_scan(wb[lane], lane);
        unsigned long long sa = wsum[0][lane], sb = wsum[1][lane];
        for (int o = 16; o > 0; o >>= 1) {
            sa += __shfl_down_sync(0xffffffffu, sa, o);
            sb += __shfl_down_sync(0xffffffffu, sb, o);
        }
        __syncwarp();
        wa[lane] = xa - wa[lane];
        wb[lane] = xb - wb[lane];
        if (lane == 0) {
            out->sum_a = sa;
            out->sum_b = sb;
            out->zero_a = nbins > 0 ? ha[0] : 0u;
            out->zero_b = nbins > 0 ? hb[0] : 0u;
        }
    }
    __syncthreads();
    ta = wa[warp] + ia - ta;                       // bins before this thread's run
    tb = wb[warp] + ib - tb;
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
    // One pass over both maps with histograms of nbins = T bins, T a power of two from 32 N_rays
    // (4096 .. 2^20); counts of T or more go to lists of room cap. The prefix sums and the K-S
    // numerator run on these bins at once: they are exact whenever the largest count is below T.
    // Otherwise the histograms are widened to the largest count and filled from the lists (or, if a
    // list ran out of room, by a second, histogram-only pass) and the K-S steps run again.
    const double nr_max = std::max(A->p.nrays_per_pix, B->p.nrays_per_pix);
    long long T = 4096;
    while (T < (1LL << 20) && (double)T < 32.0 * nr_max) T <<= 1;
    const unsigned long long cap = (unsigned long long)std::max(4096LL, n / 64);
    StatSums *d_sum = nullptr;
    unsigned *hist = nullptr, *lists = nullptr;
    long long *cum = nullptr;
    float2 *tab = nullptr;                                     // [2 T]: map a, then map b
    int rc;
    if ((rc = ctx->arena.alloc(sizeof(StatSums), (void **)&d_sum))) return rc;
    tmp.v.push_back(d_sum);
    if ((rc = ctx->arena.alloc((size_t)(2 * T) * sizeof(unsigned), (void **)&hist))) return rc;
    tmp.v.push_back(hist);
    if ((rc = ctx->arena.alloc((size_t)(2 * T) * sizeof(long long), (void **)&cum))) return rc;
    tmp.v.push_back(cum);
    if ((rc = ctx->arena.alloc((size_t)(2 * T) * sizeof(float2), (void **)&tab))) return rc;
    tmp.v.push_back(tab);
    if ((rc = ctx->arena.alloc((size_t)(2 * cap) * sizeof(unsigned), (void **)&lists))) return rc;
    tmp.v.push_back(lists);
    if ((e = cudaMemsetAsync(d_sum, 0, sizeof(StatSums), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(hist, 0, (size_t)(2 * T) * sizeof(unsigned), s)) != cudaSuccess)
        return cuda_fail(e, "memset");
    const double lra = std::log10(A->p.nrays_per_pix), lrb = std::log10(B->p.nrays_per_pix);
    // small blocks, so that the FP64 logarithms spread over many SMs
    k_log_table<<<std::max(1, std::min(4 * ctx->sms, (int)((T + 31) / 32))), 32, 0, s>>>(T, lra, lrb, tab, tab + T);
    if ((e = cudaFuncSetAttribute(k_compare, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCmpSmem)) !=
        cudaSuccess)
        return cuda_fail(e, "k_compare shared memory");
    const long long chunks = ((n / 4) * 16 + kCmpChunk - 1) / kCmpChunk;
    const int cgrid = (int)std::max(1LL, std::min((long long)(4 * ctx->sms), chunks));   // 4 CTAs fit an SM
    CmpArgs g{tab, tab + T, lra, lrb, T, hist, hist + T, lists, lists + cap, cap, 0,
              take_injection(ctx, MM_INJECT_COMPARE_NO_COPY) ? 1 : 0};
    k_compare<<<cgrid, kCmpThreads, kCmpSmem, s>>>(A->counts, B->counts, n, g, d_sum);
    auto ks_steps = [&](const unsigned *h2, long long *c2, long long nb) {
        k_scan<<<1, 1024, 0, s>>>(h2, h2 + nb, nb, c2, c2 + nb, d_sum);
        const int egrid = std::max(1, std::min(8 * ctx->sms, (int)((2 * nb + 63) / 64)));
        k_ks_eval<<<egrid, 64, 0, s>>>(h2, h2 + nb, c2, c2 + nb, nb, n, n, A->p.nrays_per_pix, B->p.nrays_per_pix,
                                        d_sum);
    };
    ks_steps(hist, cum, T);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "k_log_table/k_compare/k_scan/k_ks_eval");
    StatSums h{};
    if ((e = cudaMemcpyAsync(&h, d_sum, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "stats readback");
    if (h.fault) return fail(MM_EDEVICE, "k_compare: a copy into shared memory did not complete");
    if ((long long)h.max_count >= T) {                         // counts beyond the first histograms
        const long long nb = (long long)h.max_count + 1;
        unsigned *hist2 = nullptr;
        long long *cum2 = nullptr;
        if ((rc = ctx->arena.alloc((size_t)(2 * nb) * sizeof(unsigned), (void **)&hist2))) return rc;
        tmp.v.push_back(hist2);
        if ((rc = ctx->arena.alloc((size_t)(2 * nb) * sizeof(long long), (void **)&cum2))) return rc;
        tmp.v.push_back(cum2);
        if ((e = cudaMemsetAsync(hist2, 0, (size_t)(2 * nb) * sizeof(unsigned), s)) != cudaSuccess ||
            (e = cudaMemsetAsync(&d_sum->ks_num, 0, sizeof(long long), s)) != cudaSuccess)
            return cuda_fail(e, "memset");
        if (h.over_a <= cap && h.over_b <= cap) {
            for (int m = 0; m < 2; ++m) {
                if ((e = cudaMemcpyAsync(hist2 + m * nb, hist + m * T, (size_t)T * sizeof(unsigned),
                                         cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
                    return cuda_fail(e, "histogram copy");
                const unsigned long long cnt = m ? h.over_b : h.over_a;
                if (cnt)
                    k_list_hist<<<(int)std::min<unsigned long long>(4ULL * ctx->sms, (cnt + 255) / 256), 256, 0, s>>>(
                        lists + m * cap, cnt, hist2 + m * nb);
            }
        } else {
            CmpArgs g2{nullptr, nullptr, lra, lrb, nb, hist2, hist2 + nb, nullptr, nullptr, 0, 1, 0};
            k_compare<<<cgrid, kCmpThreads, kCmpSmem, s>>>(A->counts, B->counts, n, g2, d_sum);
        }
        ks_steps(hist2, cum2, nb);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "k_list_hist/k_compare/k_scan/k_ks_eval");
        if ((e = cudaMemcpyAsync(&h, d_sum, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(e, "stats readback");
        if (h.fault) return fail(MM_EDEVICE, "k_compare: a copy into shared memory did not complete");
    }
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

extern "C" int mm_debug_inject(mm_ctx *ctx, int32_t kind)
{
    if (!ctx) return fail(MM_EINVAL, "null context");
    if (kind != MM_INJECT_NONE && kind != MM_INJECT_COMPARE_NO_COPY && kind != MM_INJECT_DISC_NO_COPY)
        return fail(MM_EINVAL, "unknown injection");
    ctx->inject.store(kind);
    return MM_OK;
}
