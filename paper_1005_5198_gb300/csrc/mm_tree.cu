// mm_tree.cu -- the lens tree of the grouped far field (MM_FAR32 with far_group_order K > 0).
//
// The paper's tree code groups distant lenses into cells of a tree and lets a cell act
// through its multipole moments (Sect. 2.1, Eq. hierarchical). Here the tree is a quadtree
// over the lens set, built on the device once per lens set and (K, leaf size):
//   * R0 is the smallest power of two above every |x_i| and |y_i|; level L cuts
//     [-R0, R0)^2 into 2^L x 2^L cells of side s_L = 2 R0 / 2^L, and lens i lies in cell
//     (floor((x_i + R0) / s_L), floor((y_i + R0) / s_L)), each index capped at 2^L - 1 (the
//     division by a power of two is exact, so every implementation bins alike);
//   * the lenses are sorted by the Morton key of their level-16 cell (x in the even bits),
//     so that every cell of every level is a contiguous range of the sorted order; the sort
//     is a stable least-significant-digit radix sort (four passes of 8 bits);
//   * the root is the level-0 cell; a cell with more than `leaf` lenses below level 16 has
//     its non-empty quadrants of the next level as children (their key ranges are found by
//     binary search); the others are leaves;
//   * cell C has centre z_C, half-diagonal r_C = s_L / sqrt(2), mass M_C and moments
//     a_k = sum_{i in C} m_i (z_i - z_C)^k, k < K: a leaf sums its lenses (one warp per
//     leaf, lanes over lenses, a fixed reduction order), a parent shifts its children's
//     moments to its own centre, a_k = sum_child sum_{j<=k} C(k, j) a_j (z_child - z_C)^(k-j).
// Every sum has a fixed order, so the tree and its moments are the same on every run.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mm_ctx.h"
#include "mm_far.h"

namespace mm {

// Writable view of a lens tree for the kernels that build it.
struct TreeBuild {
    double r0;
    unsigned char *level;
    int *ix, *iy, *begin, *end, *first_child, *nchild;
    double2 *centre;
    double *rc, *mass;
    double2 *mom;
    const double *binom;
};

static TreeBuild build_view(const LensTree &T)
{
    return TreeBuild{T.r0, T.level, T.ix, T.iy, T.begin, T.end, T.first_child, T.nchild, T.centre, T.rc, T.mass, T.mom,
                     T.binom};
}

namespace dev {
namespace {

constexpr int kSortThreads = 256, kSortPer = 16, kSortTile = kSortThreads * kSortPer;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned spread16(unsigned v)
{
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

// Cell index of coordinate v at level L (cells of the power-of-two side s from -R0), capped.
__device__ __forceinline__ long long tree_cell(double v, double r0, double s, int level)
{
    const long long c = (long long)floor(__ddiv_rn(__dadd_rn(v, r0), s));
    const long long top = (1LL << level) - 1;
    return c < 0 ? 0 : (c > top ? top : c);
}

// Largest |x_i| or |y_i| as the bits of a non-negative double (ordered like the values).
__global__ void k_tree_absmax(const double *x, const double *y, long long n, unsigned long long *out)
{
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fmax(fabs(x[i]), fabs(y[i])));
    unsigned long long b = (unsigned long long)__double_as_longlong(m);
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(kFull, b, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, b);
}

// Morton key of each lens's level-16 cell, and the identity permutation.
__global__ void k_tree_keys(const double *x, const double *y, long long n, double r0, unsigned *keys, int *idx)
{
    const double s16 = ldexp(r0, 1 - kTreeLevels);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned ix = (unsigned)tree_cell(x[i], r0, s16, kTreeLevels);
        const unsigned iy = (unsigned)tree_cell(y[i], r0, s16, kTreeLevels);
        keys[i] = spread16(ix) | (spread16(iy) << 1);
        idx[i] = (int)i;
    }
}

// Radix pass, step 1: digit counts of every tile of kSortTile keys, digit-major:
// hist[d * tiles + t].
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const unsigned *keys, long long n, int shift,
                                                           unsigned long long *hist, long long tiles)
{
    __shared__ unsigned h[256];
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        h[threadIdx.x] = 0u;
        __syncthreads();
        const long long base = t * kSortTile;
        for (int r = 0; r < kSortPer; ++r) {
            const long long e = base + (long long)r * kSortThreads + threadIdx.x;
            if (e < n) atomicAdd(&h[(keys[e] >> shift) & 255u], 1u);
        }
        __syncthreads();
        hist[(long long)threadIdx.x * tiles + t] = h[threadIdx.x];
        __syncthreads();
    }
}

// Radix pass, step 3: stable scatter. The keys of a tile go in rounds of 256 (thread t takes
// element round * 256 + t); an element's place among the tile's keys of its digit is the
// count of that digit in earlier rounds, in earlier warps of its round and in earlier lanes
// of its warp, so equal digits keep their order.
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const unsigned *kin, const int *vin, long long n,
                                                              int shift, const unsigned long long *off,
                                                              long long tiles, unsigned *kout, int *vout)
{
    __shared__ unsigned running[256];
    __shared__ unsigned wcnt[kSortThreads / 32][256];
    const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        running[threadIdx.x] = 0u;
        for (int q = 0; q < kSortThreads / 32; ++q) wcnt[q][threadIdx.x] = 0u;
        __syncthreads();
        const long long base = t * kSortTile;
        for (int r = 0; r < kSortPer; ++r) {
            const long long e = base + (long long)r * kSortThreads + threadIdx.x;
            const bool ok = e < n;
            const unsigned key = ok ? kin[e] : 0u;
            const unsigned d = ok ? (key >> shift) & 255u : 256u;
            const unsigned peers = __match_any_sync(kFull, d);
            const unsigned before = __popc(peers & ((1u << lane) - 1u));
            if (ok && before == 0u) wcnt[w][d] = (unsigned)__popc(peers);
            __syncthreads();
            if (ok) {
                unsigned pos = running[d] + before;
                for (unsigned q = 0; q < w; ++q) pos += wcnt[q][d];
                const unsigned long long dst = off[(long long)d * tiles + t] + pos;
                kout[dst] = key;
                vout[dst] = vin[e];
            }
            __syncthreads();
            unsigned add = 0u;
            for (int q = 0; q < kSortThreads / 32; ++q) {
                add += wcnt[q][threadIdx.x];
                wcnt[q][threadIdx.x] = 0u;
            }
            running[threadIdx.x] += add;
            __syncthreads();
        }
    }
}

// First index in [b, e) whose key is >= v (keys ascending).
__device__ __forceinline__ long long lower_key(const unsigned *keys, long long b, long long e, unsigned long long v)
{
    while (b < e) {
        const long long mid = b + ((e - b) >> 1);
        if ((unsigned long long)keys[mid] < v) b = mid + 1; else e = mid;
    }
    return b;
}

// The key ranges of the four quadrants of node v: [cut[q], cut[q + 1]).
__device__ __forceinline__ void tree_quadrants(const unsigned *keys, const TreeBuild &T, int v, long long cut[5])
{
    const int L = T.level[v];
    const unsigned long long p = (unsigned long long)(spread16((unsigned)T.ix[v]) | (spread16((unsigned)T.iy[v]) << 1));
    const int sh = 2 * (kTreeLevels - L - 1);                  // key bits below the child level
    cut[0] = T.begin[v];
    cut[4] = T.end[v];
    for (int q = 1; q < 4; ++q) cut[q] = lower_key(keys, cut[q - 1], cut[4], ((p << 2) | (unsigned long long)q) << sh);
}

__device__ __forceinline__ bool tree_splits(const TreeBuild &T, int v, int leaf)
{
    return T.level[v] < kTreeLevels && T.end[v] - T.begin[v] > leaf;
}

// Non-empty children of the nodes [v0, v1) into cnt[v - v0].
__global__ void k_tree_count(const unsigned *keys, TreeBuild T, int v0, int v1, int leaf, unsigned long long *cnt)
{
    for (int v = v0 + blockIdx.x * blockDim.x + threadIdx.x; v < v1; v += gridDim.x * blockDim.x) {
        unsigned c = 0;
        if (tree_splits(T, v, leaf)) {
            long long cut[5];
            tree_quadrants(keys, T, v, cut);
            for (int q = 0; q < 4; ++q) c += cut[q + 1] > cut[q] ? 1u : 0u;
        }
        cnt[v - v0] = c;
    }
}

// Write the children of the nodes [v0, v1) from node index out0 + pos[v - v0] on, in quadrant order.
__global__ void k_tree_write(const unsigned *keys, TreeBuild T, int v0, int v1, int leaf, const unsigned long long *pos,
                             int out0)
{
    for (int v = v0 + blockIdx.x * blockDim.x + threadIdx.x; v < v1; v += gridDim.x * blockDim.x) {
        T.first_child[v] = -1;
        T.nchild[v] = 0;
        if (!tree_splits(T, v, leaf)) continue;
        long long cut[5];
        tree_quadrants(keys, T, v, cut);
        int c = out0 + (int)pos[v - v0];
        T.first_child[v] = c;
        const int L = T.level[v] + 1;
        const double s = ldexp(T.r0, 1 - L);
        for (int q = 0; q < 4; ++q) {
            if (cut[q + 1] == cut[q]) continue;
            const int ix = 2 * T.ix[v] + (q & 1), iy = 2 * T.iy[v] + (q >> 1);
            T.level[c] = (unsigned char)L;
            T.ix[c] = ix;
            T.iy[c] = iy;
            T.begin[c] = (int)cut[q];
            T.end[c] = (int)cut[q + 1];
            T.centre[c] = make_double2(__dadd_rn(-T.r0, __dmul_rn((double)ix + 0.5, s)),
                                       __dadd_rn(-T.r0, __dmul_rn((double)iy + 0.5, s)));
            T.rc[c] = __dmul_rn(s, 0.70710678118654752440);
            T.first_child[c] = -1;
            T.nchild[c] = 0;
            ++c;
        }
        T.nchild[v] = c - T.first_child[v];
    }
}

// Moments of the nodes [v0, v1) of one level, one warp per node: a leaf sums its lenses
// (lanes over lenses, a butterfly reduction per moment, lane k keeps a_k); a parent shifts
// its children's moments (lane k sums over the children in order and j ascending).
__global__ void k_tree_moments(const double *x, const double *y, const double *m, const int *perm, TreeBuild T, int v0,
                               int v1, int K)
{
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int v = v0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); v < v1; v += warps) {
        const double2 zc = T.centre[v];
        double ar = 0.0, ai = 0.0, mass = 0.0;              // lane k: a_k (k < K)
        if (T.nchild[v] == 0) {
            for (long long b = T.begin[v]; b < T.end[v]; b += 32) {
                const long long e = b + lane;
                double er = 0.0, ei = 0.0, mm = 0.0;
                if (e < T.end[v]) {
                    const int i = perm[e];
                    er = __dsub_rn(x[i], zc.x);
                    ei = __dsub_rn(y[i], zc.y);
                    mm = m ? m[i] : 1.0;
                }
                double pr = mm, pi = 0.0;                    // m e^k
                for (int k = 0; k < K; ++k) {
                    double sr = pr, si = pi;
                    for (int o = 16; o > 0; o >>= 1) {
                        sr += __shfl_xor_sync(kFull, sr, o);
                        si += __shfl_xor_sync(kFull, si, o);
                    }
                    if (lane == k) {
                        ar += sr;
                        ai += si;
                    }
                    const double nr = __dsub_rn(__dmul_rn(pr, er), __dmul_rn(pi, ei));
                    pi = __dadd_rn(__dmul_rn(pr, ei), __dmul_rn(pi, er));
                    pr = nr;
                }
                double sm = mm;
                for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(kFull, sm, o);
                mass += sm;
            }
        } else {
            for (int c = T.first_child[v]; c < T.first_child[v] + T.nchild[v]; ++c) {
                const double dr = __dsub_rn(T.centre[c].x, zc.x), di = __dsub_rn(T.centre[c].y, zc.y);
                mass += T.mass[c];
                if (lane < K) {
                    // sum_{j<=k} C(k, j) a_j(c) delta^(k-j), j from k down to 0 (delta powers ascending)
                    double pr = 1.0, pi = 0.0;
                    for (int j = lane; j >= 0; --j) {
                        const double2 a = T.mom[(long long)c * K + j];
                        const double cb = T.binom[lane * kBinomN + j];
                        ar += cb * __dsub_rn(__dmul_rn(a.x, pr), __dmul_rn(a.y, pi));
                        ai += cb * __dadd_rn(__dmul_rn(a.x, pi), __dmul_rn(a.y, pr));
                        const double nr = __dsub_rn(__dmul_rn(pr, dr), __dmul_rn(pi, di));
                        pi = __dadd_rn(__dmul_rn(pr, di), __dmul_rn(pi, dr));
                        pr = nr;
                    }
                }
            }
        }
        if (lane < K) T.mom[(long long)v * K + lane] = make_double2(ar, ai);
        if (lane == 0) T.mass[v] = mass;
    }
}

// Exclusive prefix sum of a[0 .. n) in place, a[n] = total; blocks of 1024 x 4 values
// summed first, then their totals by one CTA, then added back.
constexpr int kScanThreads = 1024, kScanPer = 4, kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ unsigned long long block_exclusive(unsigned long long v, unsigned long long *ws,
                                                              unsigned long long *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long t = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    const unsigned long long r = (w > 0 ? ws[w - 1] : 0ULL) + x - v;
    if (total) *total = ws[31];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(unsigned long long *a, long long n,
                                                             unsigned long long *tile_sum)
{
    __shared__ unsigned long long ws[32];
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanPer;
    unsigned long long v[kScanPer], s = 0;
    for (int q = 0; q < kScanPer; ++q) {
        v[q] = base + q < n ? a[base + q] : 0ULL;
        s += v[q];
    }
    unsigned long long tot;
    unsigned long long run = block_exclusive(s, ws, &tot);
    for (int q = 0; q < kScanPer; ++q) {
        if (base + q < n) a[base + q] = run;
        run += v[q];
    }
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(unsigned long long *s, long long m,
                                                            unsigned long long *total)
{
    __shared__ unsigned long long ws[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0ULL;
    __syncthreads();
    for (long long b = 0; b < m; b += kScanThreads) {
        const long long i = b + threadIdx.x;
        const unsigned long long v = i < m ? s[i] : 0ULL;
        unsigned long long tot;
        const unsigned long long r = block_exclusive(v, ws, &tot);
        if (i < m) s[i] = carry + r;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(unsigned long long *a, long long n, const unsigned long long *tile_off)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] += tile_off[i / kScanTile];
}

}  // namespace
}  // namespace dev

int scan_exclusive(mm_ctx *ctx, unsigned long long *a, long long n, cudaStream_t s)
{
    const long long tiles = std::max(1LL, (n + dev::kScanTile - 1) / dev::kScanTile);
    unsigned long long *sums = nullptr;
    int rc = ctx->arena.alloc((size_t)tiles * sizeof(unsigned long long), (void **)&sums);
    if (rc) return rc;
    dev::k_scan_tiles<<<(unsigned)tiles, dev::kScanThreads, 0, s>>>(a, n, sums);
    dev::k_scan_sums<<<1, dev::kScanThreads, 0, s>>>(sums, tiles, a + n);
    const int grid = (int)std::min<long long>((n + 255) / 256 + 1, 4096);
    dev::k_scan_add<<<grid, 256, 0, s>>>(a, n, sums);
    const cudaError_t e = cudaGetLastError();
    const cudaError_t e2 = cudaStreamSynchronize(s);       // the totals buffer goes back to the arena
    ctx->arena.free(sums);
    if (e != cudaSuccess) return cuda_fail(e, "scan");
    if (e2 != cudaSuccess) return cuda_fail(e2, "scan");
    return MM_OK;
}

void LensTree::release(DeviceArena *a)
{
    if (!a) return;
    for (void *p : {(void *)perm, (void *)level, (void *)ix, (void *)iy, (void *)begin, (void *)end, (void *)first_child,
                    (void *)nchild, (void *)centre, (void *)rc, (void *)mass, (void *)mom, (void *)binom})
        a->free(p);
    *this = LensTree{};
}

TreeView LensTree::view() const
{
    TreeView v{};
    v.r0 = r0;
    v.K = K;
    v.level = level;
    v.ix = ix;
    v.iy = iy;
    v.begin = begin;
    v.end = end;
    v.first_child = first_child;
    v.nchild = nchild;
    v.centre = centre;
    v.rc = rc;
    v.mass = mass;
    v.mom = mom;
    v.perm = perm;
    v.binom = binom;
    return v;
}

int build_lens_tree(mm_ctx *ctx, LensSet &L, int K, int leaf, cudaStream_t s)
{
    LensTree &T = L.tree;
    if (T.nodes > 0 && T.K == K && T.leaf == leaf) return MM_OK;      // cached
    T.release(&ctx->arena);
    const long long n = L.n;
    if (n <= 0) return MM_OK;
    if (n > (long long)INT32_MAX) return fail(MM_EINVAL, "grouped far field: at most 2^31 - 1 lenses");
    struct Tmp {
        DeviceArena *a;
        std::vector<void *> v;
        ~Tmp() { for (void *p : v) a->free(p); }
    } tmp{&ctx->arena, {}};
    auto talloc = [&](size_t bytes, void **out) -> int {
        int r = ctx->arena.alloc(std::max<size_t>(bytes, 16), out);
        if (!r) tmp.v.push_back(*out);
        return r;
    };
    int rc;
    // binomial coefficients for the moment shifts and the cells' series (Pascal's triangle)
    std::vector<double> binom((size_t)kBinomN * kBinomN, 0.0);
    for (int r = 0; r < kBinomN; ++r) {
        binom[(size_t)r * kBinomN] = 1.0;
        for (int k = 1; k <= r; ++k)
            binom[(size_t)r * kBinomN + k] =
                binom[(size_t)(r - 1) * kBinomN + k - 1] + (k < r ? binom[(size_t)(r - 1) * kBinomN + k] : 0.0);
    }
    // R0
    unsigned long long *d_max = nullptr;
    if ((rc = talloc(sizeof(unsigned long long), (void **)&d_max))) return rc;
    MM_CUDA(cudaMemsetAsync(d_max, 0, sizeof(unsigned long long), s));
    const int grid = (int)std::min<long long>((n + 255) / 256, 8LL * ctx->sms);
    dev::k_tree_absmax<<<grid, 256, 0, s>>>(L.dx, L.dy, n, d_max);
    unsigned long long hmax = 0;
    MM_CUDA(cudaMemcpyAsync(&hmax, d_max, sizeof(hmax), cudaMemcpyDeviceToHost, s));
    MM_CUDA(cudaStreamSynchronize(s));
    double amax;
    std::memcpy(&amax, &hmax, sizeof(amax));
    double r0 = 1.0;
    if (amax > 0.0) {
        int e;
        std::frexp(amax, &e);
        r0 = std::ldexp(1.0, e);
    }
    // keys and the stable radix sort
    unsigned *k0, *k1;
    int *v0, *v1;
    if ((rc = talloc((size_t)n * 4, (void **)&k0)) || (rc = talloc((size_t)n * 4, (void **)&k1)) ||
        (rc = ctx->arena.alloc((size_t)n * 4, (void **)&T.perm)) || (rc = talloc((size_t)n * 4, (void **)&v1)))
        return rc;
    v0 = T.perm;
    dev::k_tree_keys<<<grid, 256, 0, s>>>(L.dx, L.dy, n, r0, k0, v0);
    const long long tiles = (n + dev::kSortTile - 1) / dev::kSortTile;
    unsigned long long *hist;
    if ((rc = talloc((size_t)(256 * tiles + 1) * sizeof(unsigned long long), (void **)&hist))) return rc;
    const int sgrid = (int)std::min<long long>(tiles, 16LL * ctx->sms);
    for (int pass = 0; pass < 4; ++pass) {
        dev::k_sort_hist<<<sgrid, dev::kSortThreads, 0, s>>>(k0, n, 8 * pass, hist, tiles);
        MM_CUDA(cudaGetLastError());
        if ((rc = scan_exclusive(ctx, hist, 256 * tiles, s))) return rc;
        dev::k_sort_scatter<<<sgrid, dev::kSortThreads, 0, s>>>(k0, v0, n, 8 * pass, hist, tiles, k1, v1);
        MM_CUDA(cudaGetLastError());
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    // after four passes the sorted keys and permutation are back in k0 and T.perm
    // nodes, level by level
    long long cap = std::max(1024LL, 8 * (n / std::max(leaf, 1)) + 64);
    auto node_alloc = [&](long long c) -> int {
        LensTree U{};
        int r;
        if ((r = ctx->arena.alloc((size_t)c, (void **)&U.level)) || (r = ctx->arena.alloc((size_t)c * 4, (void **)&U.ix)) ||
            (r = ctx->arena.alloc((size_t)c * 4, (void **)&U.iy)) || (r = ctx->arena.alloc((size_t)c * 4, (void **)&U.begin)) ||
            (r = ctx->arena.alloc((size_t)c * 4, (void **)&U.end)) ||
            (r = ctx->arena.alloc((size_t)c * 4, (void **)&U.first_child)) ||
            (r = ctx->arena.alloc((size_t)c * 4, (void **)&U.nchild)) ||
            (r = ctx->arena.alloc((size_t)c * 16, (void **)&U.centre)) || (r = ctx->arena.alloc((size_t)c * 8, (void **)&U.rc))) {
            U.release(&ctx->arena);
            return r;
        }
        if (T.nodes > 0) {                                  // keep the nodes built so far
            const size_t m = (size_t)T.nodes;
            cudaMemcpyAsync(U.level, T.level, m, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(U.ix, T.ix, m * 4, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(U.iy, T.iy, m * 4, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(U.begin, T.begin, m * 4, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(U.end, T.end, m * 4, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(U.first_child, T.first_child, m * 4, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(U.nchild, T.nchild, m * 4, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(U.centre, T.centre, m * 16, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(U.rc, T.rc, m * 8, cudaMemcpyDeviceToDevice, s);
            const cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                U.release(&ctx->arena);
                return cuda_fail(e, "lens tree growth");
            }
        }
        U.perm = T.perm;
        U.binom = T.binom;
        T.perm = nullptr;
        T.binom = nullptr;
        U.nodes = T.nodes;
        U.r0 = T.r0;
        U.K = T.K;
        U.leaf = T.leaf;
        T.release(&ctx->arena);
        T = U;
        return MM_OK;
    };
    T.r0 = r0;
    T.K = K;
    T.leaf = leaf;
    if ((rc = ctx->arena.alloc(binom.size() * sizeof(double), (void **)&T.binom))) return rc;
    MM_CUDA(cudaMemcpyAsync(T.binom, binom.data(), binom.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    if ((rc = node_alloc(cap))) return rc;
    {
        const unsigned char l0 = 0;
        const int zero = 0, nn = (int)n, minus1 = -1;
        const double2 c0 = make_double2(0.0, 0.0);
        const double rc0 = 2.0 * r0 * 0.70710678118654752440;
        MM_CUDA(cudaMemcpyAsync(T.level, &l0, 1, cudaMemcpyHostToDevice, s));
        MM_CUDA(cudaMemcpyAsync(T.ix, &zero, 4, cudaMemcpyHostToDevice, s));
        MM_CUDA(cudaMemcpyAsync(T.iy, &zero, 4, cudaMemcpyHostToDevice, s));
        MM_CUDA(cudaMemcpyAsync(T.begin, &zero, 4, cudaMemcpyHostToDevice, s));
        MM_CUDA(cudaMemcpyAsync(T.end, &nn, 4, cudaMemcpyHostToDevice, s));
        MM_CUDA(cudaMemcpyAsync(T.first_child, &minus1, 4, cudaMemcpyHostToDevice, s));
        MM_CUDA(cudaMemcpyAsync(T.nchild, &zero, 4, cudaMemcpyHostToDevice, s));
        MM_CUDA(cudaMemcpyAsync(T.centre, &c0, 16, cudaMemcpyHostToDevice, s));
        MM_CUDA(cudaMemcpyAsync(T.rc, &rc0, 8, cudaMemcpyHostToDevice, s));
        MM_CUDA(cudaStreamSynchronize(s));
    }
    T.nodes = 1;
    std::vector<long long> lv{0, 1};                           // level l: nodes [lv[l], lv[l + 1])
    unsigned long long *cnt = nullptr;
    long long cnt_cap = 0;
    for (int l = 0; l < kTreeLevels; ++l) {
        const long long a = lv[(size_t)l], b = lv[(size_t)l + 1], m = b - a;
        if (m == 0) break;
        if (m + 1 > cnt_cap) {
            if (cnt) ctx->arena.free(cnt);
            cnt = nullptr;
            cnt_cap = 2 * (m + 1);
            if ((rc = ctx->arena.alloc((size_t)cnt_cap * sizeof(unsigned long long), (void **)&cnt))) return rc;
        }
        const int g = (int)std::min<long long>((m + 255) / 256, 4096);
        dev::k_tree_count<<<g, 256, 0, s>>>(k0, build_view(T), (int)a, (int)b, leaf, cnt);
        MM_CUDA(cudaGetLastError());
        if ((rc = scan_exclusive(ctx, cnt, m, s))) { ctx->arena.free(cnt); return rc; }
        unsigned long long add = 0;
        MM_CUDA(cudaMemcpyAsync(&add, cnt + m, sizeof(add), cudaMemcpyDeviceToHost, s));
        MM_CUDA(cudaStreamSynchronize(s));
        if (T.nodes + (long long)add > cap) {
            while (T.nodes + (long long)add > cap) cap *= 2;
            if (cap > (long long)INT32_MAX) { ctx->arena.free(cnt); return fail(MM_ENOMEM, "lens tree too large"); }
            if ((rc = node_alloc(cap))) { ctx->arena.free(cnt); return rc; }
        }
        dev::k_tree_write<<<g, 256, 0, s>>>(k0, build_view(T), (int)a, (int)b, leaf, cnt, (int)T.nodes);
        MM_CUDA(cudaGetLastError());
        T.nodes += (long long)add;
        lv.push_back(T.nodes);
    }
    if (cnt) ctx->arena.free(cnt);
    // moments, from the deepest level up
    if ((rc = ctx->arena.alloc((size_t)T.nodes * 8, (void **)&T.mass)) ||
        (rc = ctx->arena.alloc((size_t)T.nodes * K * 16, (void **)&T.mom)))
        return rc;
    for (int l = (int)lv.size() - 2; l >= 0; --l) {
        const long long a = lv[(size_t)l], b = lv[(size_t)l + 1];
        if (b <= a) continue;
        const int g = (int)std::min<long long>((b - a + 7) / 8, 8192);
        dev::k_tree_moments<<<g, 256, 0, s>>>(L.dx, L.dy, L.unit_mass ? nullptr : L.dm, T.perm, build_view(T), (int)a,
                                                (int)b, K);
        MM_CUDA(cudaGetLastError());
    }
    MM_CUDA(cudaStreamSynchronize(s));
    return MM_OK;
}

}  // namespace mm
