// alu_rates.cu -- measures the per-SM-clock throughput of the GB300 arithmetic
// pipes that bound the shooting kernels: scalar FFMA, packed FFMA2, MUFU
// reciprocal, DFMA, and the shooting kernel's own inner-loop instruction mixes
// run as independent chains (no memory traffic). Rates are lane-operations (or
// ray-lens interactions) per SM clock, from clock64() brackets per CTA, so they
// do not depend on the clock the GPU happens to run at; the effective clock is
// printed beside them. Output: one JSON object per line.
//
// Every loop is bounded; every store is out[gid] (gid < grid * block) or
// rec[blockIdx.x] (blockIdx.x < grid).
#include <algorithm>
#include <cstdio>
#include <vector>

#include <cuda_runtime.h>

#define CK(x)                                                                      \
    do {                                                                           \
        cudaError_t e_ = (x);                                                      \
        if (e_ != cudaSuccess) {                                                   \
            std::printf("{\"error\": \"%s: %s\"}\n", #x, cudaGetErrorString(e_));   \
            return 1;                                                              \
        }                                                                          \
    } while (0)

namespace {

__device__ __forceinline__ unsigned smid()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct Rec {
    long long t0, t1;
    unsigned sm;
};

constexpr int NCH = 8;   // independent chains per thread

// MODE 0 FFMA, 1 FFMA2, 2 MUFU rcp (x <- rcp(x) + c, not foldable), 3 DFMA,
// 4 shooting mix: lens pair per ray with a shared reciprocal (packed over lenses),
// 5 shooting mix: 3 shared : 1 two-reciprocal pair.
template <int MODE>
__global__ void kern(float *out, Rec *rec, int iters, float b, float c)
{
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    __syncthreads();
    const long long t0 = clock64();
    float a[NCH];
    double d[NCH];
    float2 p[NCH], ax[NCH], ay[NCH], ny[NCH];
    for (int k = 0; k < NCH; ++k) {
        a[k] = 1.0f + 0.001f * (threadIdx.x + k);
        d[k] = a[k];
        p[k] = make_float2(a[k], a[k] + 0.5f);
        ax[k] = ay[k] = make_float2(0.f, 0.f);
        ny[k] = make_float2(-0.01f * k - 0.001f * threadIdx.x, -0.01f * k - 0.001f * threadIdx.x);
    }
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
    float2 LX = make_float2(1.0f, 1.3f), LY = make_float2(2.0f, 1.8f);
    const float2 NX = make_float2(-0.05f, -0.05f);
    for (int it = 0; it < iters; ++it) {
        if (MODE == 4 || MODE == 5) {
            const float2 dX = __fadd2_rn(LX, NX);
            const float2 dX2 = __fmul2_rn(dX, dX);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    const float2 dY = __fadd2_rn(LY, ny[k]);
                    const float2 R2 = __ffma2_rn(dY, dY, dX2);
                    float2 W;
                    if (MODE == 4 || u < 3) {
                        const float q = rcp_approx(R2.x * R2.y);
                        W.x = q * R2.y;
                        W.y = q * R2.x;
                    } else {
                        W.x = rcp_approx(R2.x);
                        W.y = rcp_approx(R2.y);
                    }
                    ax[k] = __ffma2_rn(W, dX, ax[k]);
                    ay[k] = __ffma2_rn(W, dY, ay[k]);
                }
                LX.x += 1e-7f;
                LY.y -= 1e-7f;
            }
        } else {
#pragma unroll
            for (int k = 0; k < NCH; ++k) {
                if (MODE == 0) {
                    a[k] = fmaf(a[k], b, c); a[k] = fmaf(a[k], b, c); a[k] = fmaf(a[k], b, c); a[k] = fmaf(a[k], b, c);
                }
                if (MODE == 1) {
                    p[k] = __ffma2_rn(p[k], b2, c2); p[k] = __ffma2_rn(p[k], b2, c2);
                    p[k] = __ffma2_rn(p[k], b2, c2); p[k] = __ffma2_rn(p[k], b2, c2);
                }
                if (MODE == 2) a[k] = rcp_approx(a[k]) + c;
                if (MODE == 3) {
                    d[k] = fma(d[k], (double)b, (double)c);
                    d[k] = fma(d[k], (double)b, (double)c);
                }
            }
        }
    }
    float s = 0.f;
    for (int k = 0; k < NCH; ++k) s += a[k] + (float)d[k] + p[k].x + p[k].y + ax[k].x + ax[k].y + ay[k].x + ay[k].y;
    out[gid] = s;
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) {
        rec[blockIdx.x].t0 = t0;
        rec[blockIdx.x].t1 = t1;
        rec[blockIdx.x].sm = smid();
    }
}

// work units per thread per iteration (lane-ops, or interactions for the mixes)
const char *kNames[] = {"ffma_lane_ops", "ffma2_lane_ops", "mufu_rcp_ops", "dfma_ops", "shoot_mix_shared_pairs",
                        "shoot_mix_3to1"};
const double kUnits[] = {4.0 * NCH, 8.0 * NCH, 1.0 * NCH, 2.0 * NCH, 4.0 * NCH * 2, 4.0 * NCH * 2};
const char *kUnitName[] = {"lane-ops", "lane-ops", "ops", "ops", "interactions", "interactions"};

template <int M>
int run(int nsm, int bps, int threads, int iters, float *out, Rec *rec)
{
    const int grid = nsm * bps;
    kern<M><<<grid, threads>>>(out, rec, 4, 0.9999f, 1e-4f);
    CK(cudaDeviceSynchronize());
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0));
    kern<M><<<grid, threads>>>(out, rec, iters, 0.9999f, 1e-4f);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    std::vector<Rec> h(grid);
    CK(cudaMemcpy(h.data(), rec, grid * sizeof(Rec), cudaMemcpyDeviceToHost));
    std::vector<long long> lo(nsm, (long long)9e18), hi(nsm, 0);
    std::vector<int> cnt(nsm, 0);
    for (const Rec &r : h)
        if (r.sm < (unsigned)nsm) {
            lo[r.sm] = std::min(lo[r.sm], r.t0);
            hi[r.sm] = std::max(hi[r.sm], r.t1);
            cnt[r.sm]++;
        }
    double rate = 0, cyc = 0;
    int used = 0;
    for (int s = 0; s < nsm; ++s)
        if (cnt[s]) {
            const double c = double(hi[s] - lo[s]);
            rate += kUnits[M] * threads * (double)iters * cnt[s] / c;
            cyc += c;
            used++;
        }
    rate /= used;
    cyc /= used;
    std::printf("{\"probe\": \"%s\", \"per_sm_per_clk\": %.2f, \"unit\": \"%s\", \"effective_mhz\": %.0f, "
                "\"ctas_per_sm\": %d, \"threads\": %d}\n",
                kNames[M], rate, kUnitName[M], cyc / (ms * 1e-3) / 1e6, bps, threads);
    CK(cudaEventDestroy(e0));
    CK(cudaEventDestroy(e1));
    return 0;
}

}  // namespace

int main()
{
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, 0));
    const int nsm = prop.multiProcessorCount;
    std::printf("{\"device\": \"%s\", \"sms\": %d, \"cc\": \"%d.%d\"}\n", prop.name, nsm, prop.major, prop.minor);
    const int threads = 256, bps = 4;
    float *out = nullptr;
    Rec *rec = nullptr;
    CK(cudaMalloc(&out, (size_t)nsm * bps * threads * sizeof(float)));
    CK(cudaMalloc(&rec, (size_t)nsm * bps * sizeof(Rec)));
    int rc = 0;
    rc |= run<0>(nsm, bps, threads, 20000, out, rec);
    rc |= run<1>(nsm, bps, threads, 20000, out, rec);
    rc |= run<2>(nsm, bps, threads, 40000, out, rec);
    rc |= run<3>(nsm, bps, threads, 400, out, rec);
    rc |= run<4>(nsm, 2, threads, 2000, out, rec);
    rc |= run<5>(nsm, 2, threads, 2000, out, rec);
    CK(cudaFree(out));
    CK(cudaFree(rec));
    return rc;
}
