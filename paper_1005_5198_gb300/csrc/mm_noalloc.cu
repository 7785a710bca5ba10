// mm_noalloc.cu -- mm_shoot_noalloc: the FP32 shooting kernel for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs under another runtime or
// framework which owns the device's memory and accounts for every byte of it,
// or a tight loop where the implicit device-wide synchronisation of cudaMalloc
// and cudaFree is unacceptable. This entry point allocates nothing. The caller
// passes its own device buffers for the inputs (lens arrays) and outputs (map
// counts and totals); the kernel's scratch memory -- the FP32 tile copies of
// the lenses, the launch header, the map descriptor and the work counter --
// lives in one file-scope __device__ array of fixed size, which every GPU that
// loads this library holds until the process exits.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "mm_ctx.h"

namespace mm {
namespace {

// Capacity of the scratch array: up to this many lenses per call.
constexpr long long kNoAllocMaxLenses = 131072;
constexpr long long kNoAllocPad = (kNoAllocMaxLenses + kChunkLenses - 1) / kChunkLenses * kChunkLenses + kChunkLenses;
constexpr int kNoAllocLayout = 1;       // the default thread layout of a fresh context
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
    float4 lh[kNoAllocPad];             // (x_hi, y_hi, x_lo, y_lo), null lenses after n
    float lmf[kNoAllocPad];
    WorkHeader hdr;
    MapDesc desc;
    unsigned long long counter;
    unsigned int check;                 // checked builds: first failed bounds check of the call
};

// The scratch. In host code this name is only a stand-in for the symbol: its
// device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

std::mutex g_addr_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up on the first
// call made with that device current).
int scratch_address(int dev, NoAllocScratch **out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(MM_EINVAL, "device index beyond the no-alloc table");
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress");
        g_addr[dev] = p;
    }
    *out = static_cast<NoAllocScratch *>(g_addr[dev]);
    return MM_OK;
}

// Write the launch header and map descriptor, and zero the work counter.
__global__ void k_noalloc_setup(const WorkHeader hdr, const MapDesc desc, NoAllocScratch *sc)
{
    sc->hdr = hdr;
    sc->desc = desc;
    sc->counter = 0ULL;
    sc->check = 0u;
}

}  // namespace
}  // namespace mm

using namespace mm;

extern "C" int mm_shoot_noalloc(const double *x, const double *y, const double *m, int64_t nstar, const mm_params *p,
                                uint32_t *counts, uint64_t *totals, void *cuda_stream)
{
    Geo g;
    int rc = compute_geo(p, &g);
    if (rc) return rc;
    if (p->precision != MM_FP32C) return fail(MM_EINVAL, "mm_shoot_noalloc runs the FP32 kernel only (precision MM_FP32C)");
    if (p->ray_mode != MM_RAYS_LATTICE) return fail(MM_EINVAL, "mm_shoot_noalloc shoots lattice rays only");
    if (nstar < 0) return fail(MM_EINVAL, "nstar must be >= 0");
    if (nstar > kNoAllocMaxLenses)
        return fail(MM_EINVAL, "nstar exceeds the no-alloc scratch capacity of 131072 lenses");
    if ((nstar > 0 && (!x || !y)) || (nstar > 0 && p->mass_model != MM_MASS_UNIT && !m) || !counts || !totals)
        return fail(MM_EINVAL, "null device pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    NoAllocScratch *sc = nullptr;
    if ((rc = scratch_address(dev, &sc))) return rc;
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(e, "cudaDeviceGetAttribute");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t npix = (size_t)p->npix_side * (size_t)p->npix_side;

    // descriptor of the map, built on the host (no device memory of the library's own)
    g.nstar = nstar;
    LensSet L;                               // views into the caller's arrays and the scratch
    L.n = nstar;
    L.n_pad = (nstar + kChunkLenses - 1) / kChunkLenses * kChunkLenses + kChunkLenses;
    L.dx = const_cast<double *>(x);
    L.dy = const_cast<double *>(y);
    L.dm = const_cast<double *>(m);
    L.lh = sc->lh;
    L.lmf = sc->lmf;
    L.unit_mass = (p->mass_model == MM_MASS_UNIT);
    MapObj M;
    M.p = *p;
    M.g = g;
    M.counts = counts;
    M.totals = reinterpret_cast<unsigned long long *>(totals);
    M.lenses = std::shared_ptr<LensSet>(&L, [](LensSet *) {});
    M.variant = default_variant(L.unit_mass);   // as a fresh context chooses
    M.splits = 1;                            // no partial buffers without allocation: one CTA per tile
    M.seg_lenses = std::max<long long>(nstar, 1);
    MapDesc d;
    fill_desc(M, &d);
    d.item_begin = 0;
    d.item_first = 0;
    d.item_count = g.tiles();
    WorkHeader h{};
    h.total_work = g.tiles();
    h.n_maps = 1;

    // outputs start at zero; every piece of scratch is rewritten below
    if ((e = cudaMemsetAsync(counts, 0, npix * sizeof(uint32_t), s)) != cudaSuccess) return cuda_fail(e, "clear counts");
    if ((e = cudaMemsetAsync(totals, 0, 2 * sizeof(uint64_t), s)) != cudaSuccess) return cuda_fail(e, "clear totals");
    // the library's lens preparation, writing into the scratch (no mass array: unit masses)
    if ((e = launch_prepare_lenses(x, y, L.unit_mass ? nullptr : m, nstar, L.n_pad, sc->lh, sc->lmf, s)) != cudaSuccess)
        return cuda_fail(e, "no-alloc lens preparation");
    k_noalloc_setup<<<1, 1, 0, s>>>(h, d, sc);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "no-alloc setup");
    if (h.total_work == 0) return MM_OK;
    LaunchArgs a{};
    a.hdr = &sc->hdr;
    a.maps = &sc->desc;
    a.work_counter = &sc->counter;
    a.check = &sc->check;
    const long long cap = (long long)sms * shoot_ctas_per_sm(false, kNoAllocLayout);
    const int grid = (int)std::max(1LL, std::min((long long)h.total_work, cap));
    if ((e = launch_shoot_fp32(a, kNoAllocLayout, grid, false, false, s)) != cudaSuccess)
        return cuda_fail(e, "no-alloc shoot launch");
#ifdef MM_CHECKS
    unsigned bad = 0;                   // checked builds wait for the shoot and read its checks
    if ((e = cudaMemcpyAsync(&bad, &sc->check, sizeof(bad), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "no-alloc bounds check readback");
    if (bad) return fail(MM_EDEVICE, "bounds check failed at site " + std::to_string(bad));
#endif
    return MM_OK;
}
