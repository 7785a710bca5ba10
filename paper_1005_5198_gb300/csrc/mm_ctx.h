// mm_ctx.h -- private host-side runtime structures (context, objects, allocator).
#pragma once
#include <atomic>
#include <condition_variable>
#include <cstddef>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/mm.h"
#include "mm_far.h"
#include "mm_internal.h"

namespace mm {

// NVTX range over a host call (visible in Nsight timelines; no cost without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

// Return the library status of a failed CUDA call from the enclosing function.
#define MM_CUDA(call)                                       \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Validated geometry of a map request (host FP64).
struct Geo {
    double sigma_c, sigma_star, a, b, pix, delta, width, height, mmean, radius, mu_theory;
    long long nx, ny, nstar;
    long long i0, j0, ni, nj;
    long long tiles_x, tiles_y;
    unsigned long long tiles() const { return (unsigned long long)tiles_x * (unsigned long long)tiles_y; }
};
int compute_geo(const mm_params *p, Geo *g);

// Caching device allocator with a byte budget. Freed blocks are kept for reuse
// (size-rounded) and returned to the driver only when the budget needs room.
class DeviceArena {
public:
    void init(size_t budget) { budget_ = budget; }
    int alloc(size_t bytes, void **out);          // MM_OK / MM_ENOMEM / MM_EDEVICE
    void free(void *p);
    bool fits(size_t bytes) const;                 // could an allocation of this size succeed now
    size_t budget() const { return budget_; }
    size_t held() const { return held_; }
    void release_all();
    static size_t round(size_t bytes);
private:
    mutable std::mutex mu_;
    size_t budget_ = 0, held_ = 0;                 // held = in use + cached
    size_t live_bytes_ = 0;
    std::multimap<size_t, void *> cache_;
    std::unordered_map<void *, size_t> live_;
};

// Lens tree of a lens set for the grouped far field (mm_tree.cu), built on first use
// and kept with the set for its (K, leaf size).
struct LensTree {
    int K = 0, leaf = 0;
    double r0 = 0.0;
    long long nodes = 0;
    int *perm = nullptr;
    unsigned char *level = nullptr;
    int *ix = nullptr, *iy = nullptr, *begin = nullptr, *end = nullptr, *first_child = nullptr, *nchild = nullptr;
    double2 *centre = nullptr;
    double *rc = nullptr, *mass = nullptr;
    double2 *mom = nullptr;
    double *binom = nullptr;
    void release(DeviceArena *a);
    TreeView view() const;
};

struct LensSet {
    std::mutex tree_mu;                    // guards the tree's build (maps sharing the set)
    long long n = 0, n_pad = 0;
    double *dx = nullptr, *dy = nullptr, *dm = nullptr;
    float4 *lh = nullptr;
    float *lmf = nullptr;
    bool unit_mass = true;
    double radius = 0.0;                   // largest |x_i| of the set (the far field's density estimate)
    LensTree tree;                         // grouped far field: built on first use
    DeviceArena *arena = nullptr;
    ~LensSet();
    static size_t footprint(long long n);
};

// Lens segments per tile for a map (see kSplitTargetItems): *splits >= 1 and the
// lenses per segment, a multiple of the staging chunk.
void lens_split(const Geo &g, int precision, int *splits, long long *seg_lenses);

struct MapObj {
    mm_params p{};
    Geo g{};
    unsigned int *counts = nullptr;
    unsigned long long *totals = nullptr;   // [in, out]
    int splits = 1;                          // lens segments per tile
    long long seg_lenses = 0;
    float4 *partial = nullptr;               // split tiles: segment sums
    unsigned int *seg_done = nullptr;        // split tiles: finished segments per tile
    unsigned long long shot_total = 0;       // rays shot into the map (grows with mm_shoot_into)
    bool owns_outputs = true;                // false: counts/totals belong to another map
    // MM_FAR32: block series, near lists and the largest tail bound (mm_far.cu)
    FarDesc far{};
    float *far_coef = nullptr;
    unsigned long long *far_off = nullptr;
    int *far_idx = nullptr;
    unsigned int *far_bmax = nullptr;
    double far_bound = 0.0;
    std::shared_ptr<LensSet> lenses;
    cudaEvent_t done = nullptr;
    double seconds = 0.0;
    int variant = 0;
    DeviceArena *arena = nullptr;
    ~MapObj();
    // work items of the exact kernels and of debug dumps: tiles x lens segments (far-field
    // launches take FarDesc::items, known after far_prepare)
    unsigned long long items() const { return g.tiles() * (unsigned long long)splits; }
    static size_t footprint(const mm_params *p, const Geo &g);
};

struct Server;

struct LaunchScratch {
    WorkHeader *d_hdr = nullptr;
    MapDesc *d_maps = nullptr;
    FarDesc *d_far = nullptr;         // MM_FAR32 launches: one per map, parallel to d_maps
    unsigned long long *d_counter = nullptr;
    unsigned int *d_check = nullptr;  // checked builds: bounds-check word of the launches (LaunchArgs::check)
    int cap = 0;
    WorkHeader *h_hdr = nullptr;      // pinned
    MapDesc *h_maps = nullptr;        // pinned
    FarDesc *h_far = nullptr;         // pinned
};

}  // namespace mm

struct mm_ctx {
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    mm::DeviceArena arena;
    std::mutex mu;                                            // handle tables
    std::unordered_map<uint64_t, std::shared_ptr<mm::LensSet>> lenses;
    std::unordered_map<uint64_t, std::shared_ptr<mm::MapObj>> maps;
    std::atomic<uint64_t> next_handle{1};
    mm::LaunchScratch scratch;                                // synchronous calls
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double last_ms = 0.0;
    int last_launches = 0;
    int forced_variant = -1;
    int layout = 1;                                           // FP32 thread layout (bit-identical maps)
    std::atomic<int> inject{0};                               // one-shot test failure (mm_debug_inject)
    std::map<int, int> tuned;                                 // class key -> variant
    mm::Server *server = nullptr;
};

namespace mm {
// The test failure armed by mm_debug_inject, if it is `kind`: true once, and disarms it.
inline bool take_injection(mm_ctx *ctx, int kind)
{
    int expected = kind;
    return ctx->inject.compare_exchange_strong(expected, 0);
}
// Shared helpers used by the synchronous API and the server.
int make_lenses_from_params(mm_ctx *ctx, const mm_params *p, const Geo &g, cudaStream_t s,
                            std::shared_ptr<LensSet> *out);
int upload_lenses(mm_ctx *ctx, const double *x, const double *y, const double *m, long long n, bool unit,
                  cudaStream_t s, std::shared_ptr<LensSet> *out);
int alloc_map(mm_ctx *ctx, const mm_params *p, const Geo &g, std::shared_ptr<LensSet> lenses, cudaStream_t s,
              std::shared_ptr<MapObj> *out, const MapObj *into = nullptr);
void fill_desc(const MapObj &m, MapDesc *d);
// MM_FAR32: build the block series and near lists of map m on stream s (synchronises
// once, to size the near lists; its kernels record failed bounds checks in *check in
// checked builds); free them.
int far_prepare(mm_ctx *ctx, MapObj &m, cudaStream_t s, unsigned int *check);
// Lens tree of L for K moments and leaves of up to `leaf` lenses (kept in L.tree; rebuilt only
// for other K or leaf). Exclusive prefix sum of a[0 .. n) in place with a[n] = the total.
int build_lens_tree(mm_ctx *ctx, LensSet &L, int K, int leaf, cudaStream_t s);
int scan_exclusive(mm_ctx *ctx, unsigned long long *a, long long n, cudaStream_t s);
void far_release(MapObj &m);
// The far field's block side for parameters p, a grid g and N* lenses in a disc of the given
// radius: p.far_block, or for 0 the side that minimises the modelled time (mm_far.cu).
int far_block_for(const Geo &g, const mm_params &p, long long nstar, double radius);
// The multipole order of grouped far lenses for a map (0: no grouping): far_group_order, or for -1
// (automatic) 24 when the far field's cost model finds grouping faster (and far_order <= 16).
int far_group_for(const Geo &g, const mm_params &p, long long nstar, double radius);
int choose_variant(mm_ctx *ctx, bool unit_mass, long long nstar);
int scratch_reserve(mm_ctx *ctx, LaunchScratch *sc, int n_maps);
void scratch_free(mm_ctx *ctx, LaunchScratch *sc);
uint64_t register_map(mm_ctx *ctx, std::shared_ptr<MapObj> m);
int server_start(mm_ctx *ctx);
void server_stop(mm_ctx *ctx);
}  // namespace mm
