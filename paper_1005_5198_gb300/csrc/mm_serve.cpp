// mm_serve.cpp -- continuous-batching request loop (mm_submit / mm_poll / mm_wait).
//
// Admission: requests wait in a FIFO queue until a slot is free and their device
// footprint (lens set + map) fits the context's HBM budget. Admission workers
// (host threads with their own upload streams) then generate the seeded lens
// field, upload it and allocate the map, off the scheduler's critical path, and
// hand the request to the scheduler as "ready".
//
// Far-field maps (MM_FAR32) are served too: their workers also build the block
// series and near lists, and their work items are the far field's block rows.
//
// Scheduling: ready maps are shot in waves. A wave is one persistent launch of
// the FP32 kernel over a slice of the ray tiles of EVERY active map (plus one
// launch each for the FP64 and the far-field maps of the wave),
// replayed from a captured CUDA graph whose descriptor buffer the host rewrites
// before each replay. The slice sizes divide a work budget between the active
// maps: a priority share goes to the maps with the least work left (shortest
// remaining work first, which cuts both the median and the tail latency of a
// mixed stream), the rest evenly (processor sharing, which keeps every map
// moving). A wave always holds at least 4 tiles per CTA of the grid when the
// maps have that much work left, so maps with few tiles and many lenses cannot
// leave the GPU idle. Requests that arrive while
// waves run join the next wave, so their work overlaps on the device with the
// maps already running. Two waves are kept in flight, on two streams, so that the
// next wave's CTAs start as the current wave's last tiles drain; a map is complete
// when the wave that carried its last tile, and the wave before it, have finished. Each tile is computed
// exactly as in mm_shoot, so results are bit-identical to shooting the map alone.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "mm_ctx.h"

namespace mm {

static double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id = 0;
    mm_params p{};
    Geo g{};
    std::shared_ptr<LensSet> given;
    std::shared_ptr<MapObj> map;
    unsigned long long cursor = 0;     // next work item to schedule
    unsigned long long tiles = 0;      // work items of the map (tiles x lens segments)
    std::atomic<int> state{0};         // 0 queued, 1 admitted, 2 done, 3 failed, 4 cancelled
    bool cancel = false;               // admitted, then cancelled: stop at the next wave (under the mutex)
    double work = 0;                   // ray-lens interactions of the whole map (rays x N*)
    int err = 0;
    std::string err_msg;
    double t_submit = 0, t_admit = 0, t_done = 0;
    size_t footprint = 0;
    uint64_t map_handle = 0;
};

struct WaveItem {
    std::shared_ptr<Request> req;
    unsigned long long tiles;
    bool last;
    double work;                       // the item's share of the map's interactions
};

struct Wave {
    long long id = -1;
    int buf = 0;
    std::vector<WaveItem> items;
    unsigned long long tiles = 0;
    double interactions = 0;
    cudaEvent_t start = nullptr, end = nullptr;
};

constexpr int kAdmitWorkers = 4;

struct Server {
    mm_ctx *ctx = nullptr;
    std::thread th;
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv, done_cv, admit_cv;
    bool stop = false;
    std::deque<std::shared_ptr<Request>> queue;      // submitted, not yet admitted
    std::vector<std::shared_ptr<Request>> ready;     // prepared by a worker, not yet scheduled
    std::vector<std::shared_ptr<Request>> active;    // being shot
    int preparing = 0;                               // admitted, with a worker
    size_t reserved_bytes = 0;                       // footprint of requests being prepared
    std::unordered_map<uint64_t, std::shared_ptr<Request>> reqs;
    int max_active = 64, max_queued = 1 << 16;
    double wave_ms = 12.0;             // shorter waves cut latency, below ~8 ms the launch overhead shows
    double priority = 0.8;             // share of a wave's budget given shortest remaining work first
    cudaStream_t stream[2] = {nullptr, nullptr};     // waves alternate, so one fills the other's tail
    cudaStream_t capture = nullptr;
    cudaStream_t upload[kAdmitWorkers] = {};
    LaunchScratch sc[2], sc64[2], scfar[2];          // per wave buffer: FP32, FP64 and far-field maps
    unsigned int *far_check = nullptr;               // bounds-check word of the workers' far preparation
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [buffer][split kernel]
    int graph_cap[2][2] = {{0, 0}, {0, 0}};
    cudaEvent_t ev_start[2] = {nullptr, nullptr}, ev_end[2] = {nullptr, nullptr};
    std::deque<Wave> inflight;
    long long wave_counter = 0;
    double rate = 5.0e9;               // interactions per ms, refined from full waves
    std::atomic<uint64_t> next_id{1};
    std::string fatal;
    // counters since the server started (mm_serve_stats)
    unsigned long long n_waves = 0, n_items = 0, n_completed = 0, n_cancelled = 0, n_failed = 0;
    double work_done = 0;              // interactions of the work items of completed waves
};

static void finish(Server *S, const std::shared_ptr<Request> &r, int state, int err, const std::string &msg)
{
    (state == 2 ? S->n_completed : state == 4 ? S->n_cancelled : S->n_failed)++;
    r->err = err;
    r->err_msg = msg;
    r->t_done = now_s();
    r->state.store(state);
    S->done_cv.notify_all();
}

// Admission worker: take the head of the queue when a slot is free and its footprint
// fits, then generate/upload its lens field and allocate its map off the scheduler.
static void admit_worker(Server *S, int idx)
{
    mm_ctx *ctx = S->ctx;
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        // memory is also freed by callers releasing maps, which does not notify: re-check periodically
        while (!(S->stop || (!S->queue.empty() &&
                             (int)(S->active.size() + S->ready.size()) + S->preparing < S->max_active &&
                             ctx->arena.fits(S->reserved_bytes + S->queue.front()->footprint))))
            S->admit_cv.wait_for(lk, std::chrono::milliseconds(20));
        if (S->stop) return;
        auto r = S->queue.front();
        S->queue.pop_front();
        S->preparing++;
        S->reserved_bytes += r->footprint;
        r->t_admit = now_s();
        r->state.store(1);
        lk.unlock();
        NvtxRange nvtx_("mm serve admission");
        std::shared_ptr<LensSet> L = r->given;
        int rc = MM_OK;
        std::string msg;
        if (!L) rc = make_lenses_from_params(ctx, &r->p, r->g, S->upload[idx], &L);
        std::shared_ptr<MapObj> M;
        if (!rc) rc = alloc_map(ctx, &r->p, r->g, L, S->upload[idx], &M);
        if (!rc && r->p.precision == MM_FAR32) rc = far_prepare(ctx, *M, S->upload[idx], S->far_check);
        if (!rc) {
            const cudaError_t e = cudaStreamSynchronize(S->upload[idx]);
            if (e != cudaSuccess) rc = cuda_fail(e, "admission upload");
        }
        if (rc) msg = mm_last_error();
        lk.lock();
        S->preparing--;
        S->reserved_bytes -= r->footprint;
        if (rc) {
            finish(S, r, 3, rc, msg);
        } else {
            r->map = M;
            // work items: tiles x lens segments, or the far field's block rows
            r->tiles = r->p.precision == MM_FAR32 ? M->far.items : M->items();
            r->work = (double)r->g.ni * (double)r->g.nj * (double)L->n;
            S->ready.push_back(r);
        }
        S->cv.notify_all();
        S->admit_cv.notify_all();
    }
}

// A far-field ray costs about as much device time as this many exact interactions
// (64 ms for the 1.3e10 rays of the Fig. 1 map, against 0.185 ps per interaction).
constexpr double kFarRayInteractions = 26.0;
// An interaction of the plain FP64 kernel costs about this many of the FP32 kernel's
// (DFMA runs at 1/64 of the FP32 lane rate; measured 4.1e10 against 5.4e12 per second).
constexpr double kFp64Interactions = 130.0;

// Device time of one work item (a tile, or one lens segment of a split tile) in FP32
// interactions, or their equivalent for an FP64 tile or a far-field item (rows of tiles
// of a block).
static double tile_cost(const Request &r)
{
    if (r.p.precision == MM_FAR32)
        return (double)kTileRays * (double)r.map->far.rows_per_item * (double)r.map->far.bt * kFarRayInteractions;
    const long long n = r.map->splits > 1 ? r.map->seg_lenses : r.map->lenses->n;
    const double c = (double)kTileRays * (double)std::max(n, 8LL);
    return r.p.precision == MM_FP64 ? c * kFp64Interactions : c;
}

static int capture_graph(Server *S, int b, int split)
{
    mm_ctx *ctx = S->ctx;
    LaunchScratch *sc = &S->sc[b];
    if (S->gexec[b][split]) {
        cudaGraphExecDestroy(S->gexec[b][split]);
        S->gexec[b][split] = nullptr;
    }
    LaunchArgs a{};
    a.hdr = sc->d_hdr;
    a.maps = sc->d_maps;
    a.work_counter = sc->d_counter;
    a.check = sc->d_check;
    const int grid = ctx->sms * shoot_ctas_per_sm(false, ctx->layout);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(S->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    cudaMemcpyAsync(sc->d_hdr, sc->h_hdr, sizeof(WorkHeader), cudaMemcpyHostToDevice, S->capture);
    cudaMemcpyAsync(sc->d_maps, sc->h_maps, (size_t)sc->cap * sizeof(MapDesc), cudaMemcpyHostToDevice, S->capture);
    cudaMemsetAsync(sc->d_counter, 0, sizeof(unsigned long long), S->capture);
    launch_shoot_fp32(a, ctx->layout, grid, false, split != 0, S->capture);
    e = cudaStreamEndCapture(S->capture, &g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&S->gexec[b][split], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    S->graph_cap[b][split] = sc->cap;
    return MM_OK;
}

// Items of each map in one wave (mm_serve_plan): a `priority` share of the budget to
// the maps in increasing order of remaining work, the rest evenly, at least one item per
// map; the budget doubles until the wave holds min(min_items, all that is left).
static void plan_slices(const unsigned long long *left, const double *cost, int n, double budget, double priority,
                        unsigned long long min_items, unsigned long long *take)
{
    unsigned long long left_all = 0;
    for (int k = 0; k < n; ++k) left_all += left[k];
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return (double)left[a] * cost[a] < (double)left[b] * cost[b]; });
    for (int round = 0; round < 64; ++round) {
        unsigned long long sum = 0;
        double rest = priority * budget;
        for (int k = 0; k < n; ++k) take[k] = 0;
        for (int q = 0; q < n && rest > 0.0; ++q) {
            const int k = order[q];
            const double want = std::min(std::ceil(rest / cost[k]), 1e15);
            take[k] = std::min(left[k], (unsigned long long)want);
            rest -= (double)take[k] * cost[k];
        }
        const double even = (1.0 - priority) * budget / (double)std::max(n, 1);
        for (int k = 0; k < n; ++k) {
            const double want = std::min(std::max(1.0, std::floor(even / cost[k])), 1e15);
            take[k] = std::min(left[k], take[k] + (unsigned long long)want);
            sum += take[k];
        }
        if (sum >= std::min(min_items, left_all)) break;
        budget *= 2.0;
    }
}

// Slices of the next wave over the live maps.
static void plan_wave(Server *S, Wave *w)
{
    std::vector<std::shared_ptr<Request>> live;
    for (auto &r : S->active)
        if (r->cursor < r->tiles && !r->cancel) live.push_back(r);
    if (live.empty()) return;
    const unsigned long long min_tiles =
        4ULL * (unsigned long long)S->ctx->sms * (unsigned long long)shoot_ctas_per_sm(false, S->ctx->layout);
    const int n = (int)live.size();
    std::vector<unsigned long long> left(n), take(n);
    std::vector<double> cost(n);
    for (int k = 0; k < n; ++k) {
        left[k] = live[k]->tiles - live[k]->cursor;
        cost[k] = tile_cost(*live[k]);
    }
    plan_slices(left.data(), cost.data(), n, std::max(1.0, S->wave_ms * S->rate), S->priority, min_tiles,
                take.data());
    for (int k = 0; k < n; ++k) {
        if (!take[k]) continue;
        w->items.push_back(WaveItem{live[k], take[k], live[k]->cursor + take[k] == live[k]->tiles,
                                    live[k]->work * (double)take[k] / (double)live[k]->tiles});
        w->tiles += take[k];
        w->interactions += (double)take[k] * cost[k];
    }
}

// Write the wave's descriptors into buffer b and enqueue it on stream b.
static int launch_wave(Server *S, Wave *w)
{
    NvtxRange nvtx_("mm serve wave");
    mm_ctx *ctx = S->ctx;
    const int b = w->buf;
    int n32 = 0, n64 = 0, nfar = 0;
    for (auto &it : w->items) {
        const int pr = it.req->p.precision;
        (pr == MM_FP64 ? n64 : pr == MM_FAR32 ? nfar : n32)++;
    }
    int rc;
    if ((rc = scratch_reserve(ctx, &S->sc[b], std::max(S->max_active, n32)))) return rc;
    if (n64 && (rc = scratch_reserve(ctx, &S->sc64[b], n64))) return rc;
    if (nfar && (rc = scratch_reserve(ctx, &S->scfar[b], nfar))) return rc;
    // order: decreasing per-tile cost within each precision (large tiles first)
    std::vector<size_t> idx(w->items.size());
    for (size_t k = 0; k < idx.size(); ++k) idx[k] = k;
    std::stable_sort(idx.begin(), idx.end(),
                     [&](size_t a, size_t c) { return tile_cost(*w->items[a].req) > tile_cost(*w->items[c].req); });
    unsigned long long tot32 = 0, tot64 = 0, totfar = 0;
    int k32 = 0, k64 = 0, kfar = 0;
    for (size_t q : idx) {
        WaveItem &it = w->items[q];
        Request &r = *it.req;
        if (r.p.precision == MM_FAR32) {            // far field: its own descriptors and item range
            fill_desc(*r.map, &S->scfar[b].h_maps[kfar]);
            FarDesc &F = S->scfar[b].h_far[kfar++];
            F = r.map->far;
            F.item_begin = totfar;
            F.item_first = r.cursor;
            totfar += it.tiles;
            r.cursor += it.tiles;
            continue;
        }
        const bool fp64 = r.p.precision == MM_FP64;
        MapDesc *d = fp64 ? &S->sc64[b].h_maps[k64++] : &S->sc[b].h_maps[k32++];
        fill_desc(*r.map, d);
        d->item_first = r.cursor;
        d->item_count = it.tiles;
        d->item_begin = fp64 ? tot64 : tot32;
        (fp64 ? tot64 : tot32) += it.tiles;
        r.cursor += it.tiles;
    }
    S->sc[b].h_hdr->total_work = tot32;
    S->sc[b].h_hdr->n_maps = n32;
    cudaStream_t st = S->stream[b];
    cudaEventRecord(S->ev_start[b], st);
    if (n32) {
        int split = 0;
        for (auto &it : w->items) split |= (it.req->p.precision == MM_FP32C && it.req->map->splits > 1) ? 1 : 0;
        if (!S->gexec[b][split] || S->graph_cap[b][split] != S->sc[b].cap) {
            if ((rc = capture_graph(S, b, split))) return rc;
        }
        cudaError_t e = cudaGraphLaunch(S->gexec[b][split], st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    }
    if (n64) {
        LaunchScratch *sc = &S->sc64[b];
        sc->h_hdr->total_work = tot64;
        sc->h_hdr->n_maps = n64;
        cudaMemcpyAsync(sc->d_hdr, sc->h_hdr, sizeof(WorkHeader), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(sc->d_maps, sc->h_maps, (size_t)n64 * sizeof(MapDesc), cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(sc->d_counter, 0, sizeof(unsigned long long), st);
        LaunchArgs a{};
        a.hdr = sc->d_hdr;
        a.maps = sc->d_maps;
        a.work_counter = sc->d_counter;
        a.check = sc->d_check;
        cudaError_t e = launch_shoot_fp64(a, ctx->sms * shoot_ctas_per_sm(true, 0), false, st);
        if (e != cudaSuccess) return cuda_fail(e, "fp64 wave launch");
    }
    if (nfar) {
        LaunchScratch *sc = &S->scfar[b];
        sc->h_hdr->total_work = totfar;
        sc->h_hdr->n_maps = nfar;
        cudaMemcpyAsync(sc->d_hdr, sc->h_hdr, sizeof(WorkHeader), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(sc->d_maps, sc->h_maps, (size_t)nfar * sizeof(MapDesc), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(sc->d_far, sc->h_far, (size_t)nfar * sizeof(FarDesc), cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(sc->d_counter, 0, sizeof(unsigned long long), st);
        LaunchArgs a{};
        a.hdr = sc->d_hdr;
        a.maps = sc->d_maps;
        a.work_counter = sc->d_counter;
        a.check = sc->d_check;
        const long long grid = std::min((long long)totfar, (long long)ctx->sms * far_ctas_per_sm());
        cudaError_t e = launch_shoot_far(a, sc->d_far, totfar, (int)std::max(1LL, grid), false, st);
        if (e != cudaSuccess) return cuda_fail(e, "far-field wave launch");
    }
    cudaEventRecord(S->ev_end[b], st);
    // a finishing map may have earlier tiles in the previous wave, which runs on the
    // other stream: its completion event follows both
    bool any_last = false;
    for (auto &it : w->items) any_last = any_last || it.last;
    if (any_last && w->id > 0) cudaStreamWaitEvent(st, S->ev_end[b ^ 1], 0);
    for (auto &it : w->items)
        if (it.last) cudaEventRecord(it.req->map->done, st);
    w->start = S->ev_start[b];
    w->end = S->ev_end[b];
    return MM_OK;
}

static void complete_wave(Server *S, Wave &w, std::unique_lock<std::mutex> &lk)
{
    lk.unlock();
    cudaError_t e = cudaEventSynchronize(w.end);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, w.start, w.end);
#ifdef MM_CHECKS
    // checked builds: a failed bounds check of any wave (never reset) stops the server
    unsigned bad = 0, bad64 = 0, badfar = 0, badprep = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&bad, S->sc[w.buf].d_check, sizeof(bad), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && S->sc64[w.buf].d_check)
        e = cudaMemcpy(&bad64, S->sc64[w.buf].d_check, sizeof(bad64), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && S->scfar[w.buf].d_check)
        e = cudaMemcpy(&badfar, S->scfar[w.buf].d_check, sizeof(badfar), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&badprep, S->far_check, sizeof(badprep), cudaMemcpyDeviceToHost);
    bad64 = bad64 ? bad64 : badfar ? badfar : badprep;
#endif
    lk.lock();
    if (e != cudaSuccess) {
        S->fatal = cudaGetErrorString(e);
        for (auto &it : w.items) finish(S, it.req, 3, MM_EDEVICE, S->fatal);
        return;
    }
#ifdef MM_CHECKS
    if (bad || bad64) {
        S->fatal = "bounds check failed at site " + std::to_string(bad ? bad : bad64);
        for (auto &it : w.items) finish(S, it.req, 3, MM_EDEVICE, S->fatal);
        return;
    }
#endif
    // refine the device rate from waves large enough to fill the GPU
    const unsigned long long full = 2ULL * (unsigned long long)S->ctx->sms;
    if (ms > 0.2f && w.tiles >= full) {
        const double r = w.interactions / (double)ms;
        S->rate = std::min(2.0e10, std::max(5.0e8, 0.8 * S->rate + 0.2 * r));
    }
    S->n_waves++;
    for (auto &it : w.items) {
        S->n_items += it.tiles;
        S->work_done += it.work;
    }
    for (auto &it : w.items) {
        if (!it.last) continue;
        auto &r = it.req;
        r->map->seconds = std::max(0.0, now_s() - r->t_admit);   // admission to completion, host clock
        r->map_handle = register_map(S->ctx, r->map);
        S->active.erase(std::remove(S->active.begin(), S->active.end(), r), S->active.end());
        finish(S, r, 2, MM_OK, "");
    }
    S->admit_cv.notify_all();
}

static void loop(Server *S)
{
    mm_ctx *ctx = S->ctx;
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        if (!S->fatal.empty()) {
            for (auto &r : S->queue) finish(S, r, 3, MM_EDEVICE, S->fatal);
            S->queue.clear();
        }
        if (S->stop) {
            for (auto &r : S->queue) finish(S, r, 4, MM_ECANCELED, "server stopped");
            S->queue.clear();
        }
        for (auto &r : S->ready) {
            if (r->cancel) finish(S, r, 4, MM_ECANCELED, "cancelled");    // prepared, never shot
            else S->active.push_back(r);
        }
        S->ready.clear();
        // cancelled maps leave once no wave in flight holds their tiles
        for (size_t k = 0; k < S->active.size();) {
            auto r = S->active[k];
            bool held = false;
            for (auto &w : S->inflight)
                for (auto &it : w.items) held = held || it.req == r;
            if (r->cancel && !held) {
                S->active.erase(S->active.begin() + (long)k);
                finish(S, r, 4, MM_ECANCELED, "cancelled");
                S->admit_cv.notify_all();
            } else {
                ++k;
            }
        }
        bool have_work = false;
        for (auto &r : S->active) have_work = have_work || (r->cursor < r->tiles && !r->cancel);
        if (S->stop && S->inflight.empty() && !have_work && S->preparing == 0) {
            for (auto &r : S->active) finish(S, r, 4, MM_ECANCELED, "server stopped");
            S->active.clear();
            break;
        }
        if (have_work && S->inflight.size() < 2 && S->fatal.empty()) {
            Wave w;
            w.buf = (int)(S->wave_counter & 1);
            w.id = S->wave_counter++;
            plan_wave(S, &w);
            int rc = launch_wave(S, &w);
            if (rc) {
                S->fatal = mm_last_error();
                for (auto &it : w.items) finish(S, it.req, 3, rc, S->fatal);
                continue;
            }
            S->inflight.push_back(std::move(w));
            continue;
        }
        if (!S->inflight.empty()) {
            Wave w = std::move(S->inflight.front());
            S->inflight.pop_front();
            complete_wave(S, w, lk);
            continue;
        }
        S->cv.wait_for(lk, std::chrono::milliseconds(20));
    }
}

int server_start(mm_ctx *ctx)
{
    if (ctx->server) return MM_OK;
    auto *S = new Server();
    S->ctx = ctx;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaStreamCreateWithFlags(&S->stream[0], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->stream[1], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->capture, cudaStreamNonBlocking);
    for (int k = 0; k < kAdmitWorkers && e == cudaSuccess; ++k)
        e = cudaStreamCreateWithFlags(&S->upload[k], cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaEventCreate(&S->ev_start[b]);
        if (e == cudaSuccess) e = cudaEventCreate(&S->ev_end[b]);
    }
    if (e == cudaSuccess) e = cudaMalloc(&S->far_check, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(S->far_check, 0, sizeof(unsigned int));
    if (e != cudaSuccess) {
        delete S;
        return cuda_fail(e, "server streams/events");
    }
    ctx->server = S;
    S->th = std::thread(loop, S);
    for (int k = 0; k < kAdmitWorkers; ++k) S->workers.emplace_back(admit_worker, S, k);
    return MM_OK;
}

void server_stop(mm_ctx *ctx)
{
    Server *S = ctx->server;
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    S->admit_cv.notify_all();
    for (auto &t : S->workers)
        if (t.joinable()) t.join();
    if (S->th.joinable()) S->th.join();
    cudaStreamSynchronize(S->stream[0]);
    cudaStreamSynchronize(S->stream[1]);
    for (int b = 0; b < 2; ++b) {
        for (int k = 0; k < 2; ++k)
            if (S->gexec[b][k]) cudaGraphExecDestroy(S->gexec[b][k]);
        scratch_free(ctx, &S->sc[b]);
        scratch_free(ctx, &S->sc64[b]);
        scratch_free(ctx, &S->scfar[b]);
        cudaEventDestroy(S->ev_start[b]);
        cudaEventDestroy(S->ev_end[b]);
    }
    if (S->far_check) cudaFree(S->far_check);
    cudaStreamDestroy(S->stream[0]);
    cudaStreamDestroy(S->stream[1]);
    cudaStreamDestroy(S->capture);
    for (int k = 0; k < kAdmitWorkers; ++k) cudaStreamDestroy(S->upload[k]);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->reqs.clear();
    }
    delete S;
    ctx->server = nullptr;
}

static std::shared_ptr<Request> find_req(Server *S, mm_req id)
{
    auto it = S->reqs.find(id);
    return it == S->reqs.end() ? nullptr : it->second;
}

}  // namespace mm

using namespace mm;

extern "C" {

int mm_serve_config(mm_ctx *ctx, int32_t max_active, int32_t max_queued, double wave_ms)
{
    if (!ctx || max_active < 0 || max_queued < 0 || !(wave_ms >= 0.0)) return fail(MM_EINVAL, "bad serve config");
    int rc = server_start(ctx);
    if (rc) return rc;
    Server *S = ctx->server;
    std::lock_guard<std::mutex> lk(S->mu);
    if (max_active) S->max_active = max_active;
    if (max_queued) S->max_queued = max_queued;
    if (wave_ms > 0.0) S->wave_ms = wave_ms;
    S->admit_cv.notify_all();
    return MM_OK;
}

int mm_serve_priority(mm_ctx *ctx, double priority_share)
{
    if (!ctx || !(priority_share >= 0.0 && priority_share <= 1.0)) return fail(MM_EINVAL, "priority share outside [0, 1]");
    int rc = server_start(ctx);
    if (rc) return rc;
    Server *S = ctx->server;
    std::lock_guard<std::mutex> lk(S->mu);
    S->priority = priority_share;
    return MM_OK;
}

int mm_serve_plan(const uint64_t *left, const double *cost, int32_t n, double budget, double priority_share,
                  uint64_t min_items, uint64_t *take)
{
    if (n < 0 || (n > 0 && (!left || !cost || !take)) || !(budget > 0.0) ||
        !(priority_share >= 0.0 && priority_share <= 1.0))
        return fail(MM_EINVAL, "bad plan arguments");
    for (int k = 0; k < n; ++k)
        if (!(cost[k] > 0.0) || !std::isfinite(cost[k])) return fail(MM_EINVAL, "work item cost must be positive");
    static_assert(sizeof(unsigned long long) == sizeof(uint64_t), "item counts are 64-bit");
    plan_slices(reinterpret_cast<const unsigned long long *>(left), cost, n, budget, priority_share, min_items,
                reinterpret_cast<unsigned long long *>(take));
    return MM_OK;
}

int mm_submit(mm_ctx *ctx, mm_lenses lenses, const mm_params *p, mm_req *out)
{
    if (!ctx || !out) return fail(MM_EINVAL, "null argument");
    auto r = std::make_shared<Request>();
    int rc = compute_geo(p, &r->g);
    if (rc) return rc;
    if (p->ray_mode != MM_RAYS_LATTICE) return fail(MM_EINVAL, "mm_submit serves lattice rays only");
    r->p = *p;
    if (lenses) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->lenses.find(lenses);
        if (it == ctx->lenses.end()) return fail(MM_ENOTFOUND, "unknown lens set");
        r->given = it->second;
        r->g.nstar = r->given->n;
    }
    r->footprint = MapObj::footprint(p, r->g) + (r->given ? 0 : LensSet::footprint(r->g.nstar));
    if (r->footprint > ctx->arena.budget()) return fail(MM_ENOMEM, "request footprint exceeds the HBM budget");
    if ((rc = server_start(ctx))) return rc;
    Server *S = ctx->server;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if ((int)S->queue.size() >= S->max_queued) return fail(MM_EBUSY, "request queue full");
        r->id = S->next_id.fetch_add(1);
        r->t_submit = now_s();
        S->queue.push_back(r);
        S->reqs[r->id] = r;
    }
    S->admit_cv.notify_one();
    *out = r->id;
    return MM_OK;
}

int mm_poll(mm_ctx *ctx, mm_req req, int *done, mm_map *map_out)
{
    if (!ctx || !done) return fail(MM_EINVAL, "null argument");
    Server *S = ctx->server;
    if (!S) return fail(MM_ENOTFOUND, "unknown request");
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r = find_req(S, req);
    }
    if (!r) return fail(MM_ENOTFOUND, "unknown request");
    const int st = r->state.load();
    *done = 0;
    if (st == 2) {
        *done = 1;
        if (map_out) *map_out = r->map_handle;
        return MM_OK;
    }
    if (st == 3) {
        *done = 1;
        return fail(r->err, r->err_msg);
    }
    if (st == 4) {
        *done = 1;
        return fail(MM_ECANCELED, "request cancelled");
    }
    return MM_OK;
}

int mm_wait(mm_ctx *ctx, mm_req req, int64_t timeout_ns, mm_map *map_out)
{
    if (!ctx) return fail(MM_EINVAL, "null context");
    Server *S = ctx->server;
    if (!S) return fail(MM_ENOTFOUND, "unknown request");
    std::unique_lock<std::mutex> lk(S->mu);
    auto r = find_req(S, req);
    if (!r) return fail(MM_ENOTFOUND, "unknown request");
    auto pred = [&] { return r->state.load() >= 2; };
    if (timeout_ns < 0) S->done_cv.wait(lk, pred);
    else if (!S->done_cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns), pred))
        return fail(MM_ETIMEDOUT, "request still running");
    const int st = r->state.load();
    if (st == 2) {
        if (map_out) *map_out = r->map_handle;
        return MM_OK;
    }
    if (st == 4) return fail(MM_ECANCELED, "request cancelled");
    return fail(r->err, r->err_msg);
}

int mm_cancel(mm_ctx *ctx, mm_req req)
{
    if (!ctx) return fail(MM_EINVAL, "null context");
    Server *S = ctx->server;
    if (!S) return fail(MM_ENOTFOUND, "unknown request");
    std::lock_guard<std::mutex> lk(S->mu);
    auto r = find_req(S, req);
    if (!r) return fail(MM_ENOTFOUND, "unknown request");
    auto it = std::find(S->queue.begin(), S->queue.end(), r);
    if (it != S->queue.end()) {
        S->queue.erase(it);
        finish(S, r, 4, MM_ECANCELED, "cancelled");
        return MM_OK;
    }
    // admitted: stops before its next work item is scheduled, unless all of it is on the GPU
    if (r->state.load() != 1 || r->cancel || (r->tiles > 0 && r->cursor >= r->tiles))
        return fail(MM_EBUSY, "request already finished or fully scheduled");
    r->cancel = true;
    S->cv.notify_all();
    return MM_OK;
}

int mm_serve_stats(mm_ctx *ctx, mm_serve_stats_t *out)
{
    if (!ctx || !out) return fail(MM_EINVAL, "null argument");
    std::memset(out, 0, sizeof(*out));
    Server *S = ctx->server;
    if (!S) return MM_OK;
    std::lock_guard<std::mutex> lk(S->mu);
    out->waves = S->n_waves;
    out->items = S->n_items;
    out->interactions = S->work_done;
    out->completed = S->n_completed;
    out->cancelled = S->n_cancelled;
    out->failed = S->n_failed;
    out->queued = (int32_t)S->queue.size();
    out->preparing = S->preparing;
    out->active = (int32_t)(S->active.size() + S->ready.size());
    return MM_OK;
}

int mm_req_times(mm_ctx *ctx, mm_req req, double *t_queue, double *t_total)
{
    if (!ctx) return fail(MM_EINVAL, "null context");
    Server *S = ctx->server;
    if (!S) return fail(MM_ENOTFOUND, "unknown request");
    std::lock_guard<std::mutex> lk(S->mu);
    auto r = find_req(S, req);
    if (!r) return fail(MM_ENOTFOUND, "unknown request");
    if (r->state.load() < 2) return fail(MM_EAGAIN, "request not finished");
    if (t_queue) *t_queue = (r->t_admit > 0 ? r->t_admit : r->t_done) - r->t_submit;
    if (t_total) *t_total = r->t_done - r->t_submit;
    return MM_OK;
}

}  // extern "C"
