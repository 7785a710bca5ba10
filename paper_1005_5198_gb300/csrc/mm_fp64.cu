// mm_fp64.cu -- the plain FP64 shooting kernel, the lens-preparation kernel and
// the launch dispatch for the FP32 thread layouts.
//
// FP64 path (MM_FP64): the same 64 x 32-ray tiles and persistent loop as the
// FP32 kernel, every operation in FP64 and lenses summed in index order: for
// each ray, alpha = sum_i m_i (x - x_i)/|x - x_i|^2 (Sect. 2, Eq. sigma), then
// y1 = (1 - gamma) x1 - sigma_c x1 - alpha1, y2 = (1 + gamma) x2 - sigma_c x2 -
// alpha2 and pixel floor((y + L/2) / p). This is the plain form the FP32 path
// is compared with.
#include "mm_device.cuh"

namespace mm {

cudaError_t launch_fp32_layout0(const LaunchArgs &, int, bool, bool, cudaStream_t);
cudaError_t launch_fp32_layout1(const LaunchArgs &, int, bool, bool, cudaStream_t);
cudaError_t launch_fp32_layout2(const LaunchArgs &, int, bool, bool, cudaStream_t);
cudaError_t launch_fp32_layout3(const LaunchArgs &, int, bool, bool, cudaStream_t);

namespace dev {
namespace {

constexpr int K64 = 8;   // rays per thread (one column, 8 rows), 256 threads per 64 x 32 tile

// One lens's term of the deflection sum for one ray (Eq. sigma), with every rounding
// fixed (explicit FP64 intrinsics), so that the map kernel and the ray-list kernel below
// compute each ray identically. A ray exactly on a lens sets `on` and adds nothing.
__device__ __forceinline__ void fp64_term(double x1, double x2, double2 L, double m, double &a1, double &a2, bool &on)
{
    const double d1 = __dsub_rn(x1, L.x), d2 = __dsub_rn(x2, L.y);
    const double r2 = __fma_rn(d1, d1, __dmul_rn(d2, d2));
    if (r2 == 0.0) {
        on = true;
    } else {
        const double t = __ddiv_rn(m, r2);
        a1 = __fma_rn(t, d1, a1);
        a2 = __fma_rn(t, d2, a2);
    }
}

// Lattice coordinate of ray index g along one axis: (g + 1/2 - n/2) delta.
__device__ __forceinline__ double fp64_lattice(long long g, double half_n, double delta)
{
    return __dmul_rn(__dsub_rn(__dadd_rn((double)g, 0.5), half_n), delta);
}

// Lens equation and pixel (Eq. sigma, then floor((y + L/2) / p) per axis): the flat
// pixel index, or -1 when the ray lands outside the map or is not finite.
__device__ __forceinline__ long long fp64_pixel(const MapDesc &M, double x1, double x2, double a1, double a2)
{
    const double y1 = __dsub_rn(__fma_rn(M.one_m_gamma, x1, -__dmul_rn(M.sigma_c, x1)), a1);
    const double y2 = __dsub_rn(__fma_rn(M.one_p_gamma, x2, -__dmul_rn(M.sigma_c, x2)), a2);
    const double u1 = floor(__ddiv_rn(__dadd_rn(y1, M.half_side), M.pix));
    const double u2 = floor(__ddiv_rn(__dadd_rn(y2, M.half_side), M.pix));
    const double nsd = (double)M.nside;
    if (!(u1 >= 0.0 && u1 < nsd && u2 >= 0.0 && u2 < nsd)) return -1;
    return (long long)u2 * (long long)M.nside + (long long)u1;
}

template <bool DUMP>
__device__ void tile_fp64(const LaunchArgs &A, const MapDesc &M, unsigned long long tile, int item, SmemFP64 &S,
                          unsigned &cnt_in, unsigned &cnt_out)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int w = tid >> 5;
    const int iloc = (w & 1) * 32 + lane;
    const int jloc0 = (w >> 1) * K64;
    const long long tx = (long long)(tile % (unsigned long long)M.tiles_x);
    const long long ty = (long long)(tile / (unsigned long long)M.tiles_x);
    const long long ib = M.i0 + tx * kTileX;
    const long long jb = M.j0 + ty * kTileY;
    const long long gi = ib + iloc;
    double x1[K64], x2[K64], a1[K64], a2[K64];
    bool on[K64];
#pragma unroll
    for (int r = 0; r < K64; ++r) {
        if (M.random_rays) {                          // random rays: each at its own place in the tile
            float fx, fy;
            random_cell(M, gi, jb + jloc0 + r, fx, fy);
            x1[r] = random_coord(ib, fx, M.half_nx, M.delta);
            x2[r] = random_coord(jb, fy, M.half_ny, M.delta);
        } else {
            x1[r] = fp64_lattice(gi, M.half_nx, M.delta);
            x2[r] = fp64_lattice(jb + jloc0 + r, M.half_ny, M.delta);
        }
        a1[r] = a2[r] = 0.0;
        on[r] = false;
    }
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
            const double2 Lp = S.lens64[k];
            const double m = S.m64[k];
#pragma unroll
            for (int r = 0; r < K64; ++r) fp64_term(x1[r], x2[r], Lp, m, a1[r], a2[r], on[r]);
        }
    }
    const bool col_ok = gi < M.i0 + M.ni;
#pragma unroll
    for (int r = 0; r < K64; ++r) {
        const long long gj = jb + jloc0 + r;
        const long long px = fp64_pixel(M, x1[r], x2[r], a1[r], a2[r]);
        const bool valid = col_ok && gj < M.j0 + M.nj;
        const bool inside = valid && !on[r] && px >= 0;
        const unsigned pix = inside ? (unsigned)px : 0xffffffffu;
        emit_ray<DUMP>(A, M, item, iloc + kTileX * (jloc0 + r), valid, inside, pix, a1[r], a2[r], cnt_in, cnt_out);
    }
}

template <bool DUMP>
__global__ void __launch_bounds__(256, 1) k_shoot_fp64(const LaunchArgs A)
{
    __shared__ SmemFP64 S;
    persistent_loop<DUMP>(A, S.loop, [&](const MapDesc &M, unsigned long long tile, int, int item, unsigned &ci,
                                          unsigned &co) { tile_fp64<DUMP>(A, M, tile, item, S, ci, co); });
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
            lmf[k] = m ? __double2float_rn(m[k]) : 1.0f;     // no mass array: unit masses
        } else {
            lh[k] = make_float4(kNullX, 0.f, 0.f, 0.f);
            lmf[k] = 0.f;
        }
    }
}

// Rays of a list (global lattice indices), one thread each, through the map kernel's
// per-ray FP64 arithmetic (fp64_lattice, fp64_term in lens order, fp64_pixel): each ray's
// deflection and pixel equal the ones the FP64 map kernel computes for it, at the cost of
// that ray alone rather than of its whole tile. Lenses are staged through shared memory
// in chunks of 256, as in the map kernel.
__global__ void __launch_bounds__(256) k_rays_fp64(const MapDesc M, const long long *ri, const long long *rj,
                                                   long long n, double *alpha, long long *pixel)
{
    __shared__ double2 lens64[kChunkPairs];
    __shared__ double m64[kChunkPairs];
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool act = k < n;
    double x1 = act ? fp64_lattice(ri[k], M.half_nx, M.delta) : 0.0;
    double x2 = act ? fp64_lattice(rj[k], M.half_ny, M.delta) : 0.0;
    if (act && M.random_rays) {                       // the ray's tile starts at cell (64 Ti, 32 Tj)
        float fx, fy;
        random_cell(M, ri[k], rj[k], fx, fy);
        x1 = random_coord(ri[k] / kTileX * kTileX, fx, M.half_nx, M.delta);
        x2 = random_coord(rj[k] / kTileY * kTileY, fy, M.half_ny, M.delta);
    }
    double a1 = 0.0, a2 = 0.0;
    bool on = false;
    for (long long base = 0; base < M.nstar; base += kChunkPairs) {
        __syncthreads();
        const long long g = base + threadIdx.x;
        if (g < M.nstar) {
            lens64[threadIdx.x] = make_double2(M.lx[g], M.ly[g]);
            m64[threadIdx.x] = M.lm[g];
        }
        __syncthreads();
        const int c = (int)min((long long)kChunkPairs, M.nstar - base);
        if (act)
            for (int q = 0; q < c; ++q) fp64_term(x1, x2, lens64[q], m64[q], a1, a2, on);
    }
    if (act) {
        alpha[2 * k] = a1;
        alpha[2 * k + 1] = a2;
        pixel[k] = on ? -1LL : fp64_pixel(M, x1, x2, a1, a2);
    }
}

}  // namespace
}  // namespace dev

cudaError_t launch_prepare_lenses(const double *x, const double *y, const double *m, long long n, long long n_pad,
                                  float4 *lh, float *lmf, cudaStream_t s)
{
    if (n_pad <= 0) return cudaSuccess;
    const int grid = (int)min((n_pad + 255) / 256, (long long)4096);
    dev::k_prepare_lenses<<<grid, 256, 0, s>>>(x, y, m, n, n_pad, lh, lmf);
    return cudaGetLastError();
}

cudaError_t launch_rays_fp64(const MapDesc &M, const long long *ri, const long long *rj, long long n, double *alpha,
                             long long *pixel, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    dev::k_rays_fp64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(M, ri, rj, n, alpha, pixel);
    return cudaGetLastError();
}

cudaError_t launch_shoot_fp32(const LaunchArgs &args, int layout, int grid, bool dump, bool split, cudaStream_t s)
{
    switch (layout) {
    case 1: return launch_fp32_layout1(args, grid, dump, split, s);
    case 2: return launch_fp32_layout2(args, grid, dump, split, s);
    case 3: return launch_fp32_layout3(args, grid, dump, split, s);
    default: return launch_fp32_layout0(args, grid, dump, split, s);
    }
}

cudaError_t launch_shoot_fp64(const LaunchArgs &args, int grid, bool dump, cudaStream_t s)
{
    if (dump) dev::k_shoot_fp64<true><<<grid, 256, 0, s>>>(args);
    else dev::k_shoot_fp64<false><<<grid, 256, 0, s>>>(args);
    return cudaGetLastError();
}

// Per layout: threads per CTA and CTAs per SM (must match mm_fp32_*.cu).
static const int kLayoutThreads[kNumLayouts] = {256, 256, 128, 256};
static const int kLayoutCtas[kNumLayouts] = {2, 2, 2, 1};

int shoot_ctas_per_sm(bool fp64, int layout)
{
    if (fp64) return 1;
    return (layout >= 0 && layout < kNumLayouts) ? kLayoutCtas[layout] : 2;
}

int layout_threads(int layout) { return (layout >= 0 && layout < kNumLayouts) ? kLayoutThreads[layout] : 256; }

const char *layout_name(int layout)
{
    static const char *names[kNumLayouts] = {
        "1 column x 8 rows per thread, sums in registers, 256 threads x 2 CTAs/SM",
        "2 columns x 4 rows per thread, sums in registers, 256 threads x 2 CTAs/SM",
        "2 columns x 8 rows per thread, sums in shared memory, 128 threads x 2 CTAs/SM",
        "2 columns x 4 rows per thread, sums in registers, 256 threads x 1 CTA/SM"};
    return (layout >= 0 && layout < kNumLayouts) ? names[layout] : "invalid";
}

const char *variant_name(int v)
{
    static const char *names[kNumVariants] = {"shared-rcp 3/4, fold 64", "shared-rcp 3/4, fold 32",
                                              "shared-rcp 2/4, fold 64", "shared-rcp 4/4, fold 64"};
    return (v >= 0 && v < kNumVariants) ? names[v] : "invalid";
}

}  // namespace mm
