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
    const double x1 = ((double)gi + 0.5 - M.half_nx) * M.delta;
    double x2[K64], a1[K64], a2[K64];
#pragma unroll
    for (int r = 0; r < K64; ++r) {
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
            const double2 Lp = S.lens64[k];
            const double m = S.m64[k];
#pragma unroll
            for (int r = 0; r < K64; ++r) {
                const double d1 = x1 - Lp.x, d2 = x2[r] - Lp.y;
                const double r2 = d1 * d1 + d2 * d2;
                if (r2 == 0.0) {
                    onlens |= 1u << r;
                } else {
                    const double t = m / r2;
                    a1[r] += t * d1;
                    a2[r] += t * d2;
                }
            }
        }
    }
    const bool col_ok = gi < M.i0 + M.ni;
    const double nsd = (double)M.nside;
#pragma unroll
    for (int r = 0; r < K64; ++r) {
        const long long gj = jb + jloc0 + r;
        const double y1 = M.one_m_gamma * x1 - M.sigma_c * x1 - a1[r];
        const double y2 = M.one_p_gamma * x2[r] - M.sigma_c * x2[r] - a2[r];
        const double u1 = floor((y1 + M.half_side) / M.pix);
        const double u2 = floor((y2 + M.half_side) / M.pix);
        const bool valid = col_ok && gj < M.j0 + M.nj;
        const bool inside = valid && !((onlens >> r) & 1u) && u1 >= 0.0 && u1 < nsd && u2 >= 0.0 && u2 < nsd;
        const unsigned pix = inside ? (unsigned)u2 * (unsigned)M.nside + (unsigned)u1 : 0xffffffffu;
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
