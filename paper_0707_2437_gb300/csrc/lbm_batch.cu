// Host side of the batched form (the kernels are in lbm_batch_kernels.cuh):
// many uneven grids (any size, tau, c2 and storage) advanced by
// one persistent cooperative kernel over a tile work-list, with a grid-wide
// barrier between time steps, replayed from a CUDA graph.
//
// Work-list: every grid is cut into tiles of (32*vec columns) x (rows rows),
// one warp per tile per step; within a step the resident warps take tiles in
// list order from an atomic counter.  Within a time step tiles are independent (each reads its grid's
// input buffer and writes the other one); between steps every block waits at
// a barrier, because a tile's pull reaches two rows and one column into its
// neighbours and its store overwrites what they read one step earlier.
//
// Every barrier wait is bounded (wall-clock limit read from %globaltimer): a
// block that gives up sets a status word and returns, all other blocks see the
// status at their next barrier and return too, so the kernel always ends.
#include <algorithm>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"
#include "lbm_batch_kernels.cuh"

struct lbm_batch {
    std::vector<lbm_grid *> grids;
    // Per grid, the c2 field pointer and rounding mode the work-list was built
    // for (a change rebuilds it at the next step call).
    std::vector<const float *> built_a15f;
    std::vector<int> built_rounding;
    cudaStream_t stream = nullptr;
    int device = 0;
    int rows = 16;
    bool fit_rows = true;   // default: lockstep work-lists may use shorter tiles
    int lock_rows = 16;     // tile height of the lockstep work-list as built
    int blocks_per_sm = 0;  // 0: the occupancy limit
    // Kind groups: consecutive ranges of the tile list, each run by its own
    // persistent launch (a specialised k_batch_one, or k_batch for the rest),
    // one after the other on the batch's stream.
    struct Group {
        int begin = 0, count = 0;
        BatchKernel kernel = nullptr;
        FlowKernel fkernel = nullptr;  // flow schedule
        int max_blocks_per_sm = 1;
    };
    std::vector<Group> groups;
    int walk16 = LBM_WALK16_AUTO;  // walk of 16-bit grids (lbm_batch_set_walk16)
    int sms = 1;
    unsigned long long timeout_ns = 1000000000ULL;
    // device
    GridDesc *d_grids = nullptr;
    Tile *d_tiles = nullptr;
    int ntiles = 0;
    long long *d_limit = nullptr;
    int *d_parity = nullptr;
    uint32_t *d_t0 = nullptr;
    unsigned *d_bar = nullptr;
    int *d_status = nullptr;
    // pinned host mirrors of the per-call arrays
    long long *h_limit = nullptr;
    int *h_parity = nullptr;
    uint32_t *h_t0 = nullptr;
    int *h_status = nullptr;
    cudaEvent_t copied = nullptr;  // the per-call arrays have been read
    // Streams of members other than the batch's own (as of the last step
    // call), with one event each, and the event that marks the batch's work.
    std::vector<cudaStream_t> xs;
    std::vector<cudaEvent_t> xev;
    cudaEvent_t done = nullptr;
    // graph cache (one step count)
    cudaGraphExec_t graph = nullptr;
    long long graph_n = -1;
    // Launch mode (lbm_batch_set_launch): LBM_LAUNCH_AUTO tries a graph and
    // falls back to direct launches if capture fails, LBM_LAUNCH_GRAPH
    // requires the graph, LBM_LAUNCH_DIRECT never captures.  `capture_failed`
    // records an AUTO fallback; `last_launch` is how the last step call ran
    // (0 before the first one).
    int launch_mode = LBM_LAUNCH_AUTO;
    bool capture_failed = false;
    int last_launch = 0;
    // Schedule (lbm_batch_set_schedule): lockstep kind groups, or one flow
    // launch over all grids with per-tile progress (control words per grid,
    // completed steps per tile, and the count of grids with work this call).
    int schedule = LBM_SCHEDULE_LOCKSTEP;
    unsigned long long *d_ctl = nullptr;
    int *d_prog = nullptr;
    size_t prog_cap = 0;
    int *d_nwork = nullptr;
    int *h_nwork = nullptr;
    // Paired tiles (split walk) in the lockstep work-list.
    int paired = 0;
};

static int bfail(int code, const std::string &m) {
    set_error(m);
    return code;
}

static int bcuda(cudaError_t e, const char *where) {
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
}

#define BCK(call)                                           \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return bcuda(e_, #call);     \
    } while (0)

static void drop_graph(lbm_batch *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_n = -1;
}

// Sites per lane of a grid's walk.  FP32: 4 (128-bit loads) when nx is a
// multiple of 4.  16-bit: 8 (128-bit loads, rows and any c2 field's values
// through shared memory) when nx is a multiple of 8 and the walk is
// LBM_WALK16_AUTO or LBM_WALK16_V8; else 4 (64-bit loads, one row prefetched
// in registers) when nx is a multiple of 4.  Any other nx: 1.  (Measured on GB300: 8 sites
// per lane run 15 % faster than 4 with nearest rounding and 10 % faster with
// stochastic rounding.)
static int batch_vec(const lbm_batch *b, const lbm_grid *g) {
    const bool eight = b->walk16 == LBM_WALK16_V8 || b->walk16 == LBM_WALK16_AUTO;
    if (g->storage != ST_F32 && eight && g->nx % 8 == 0) return 8;
    return g->nx % 4 == 0 ? 4 : 1;
}

// Copies the grid table and the tile list to the device.
static int upload_worklist(lbm_batch *b, const std::vector<GridDesc> &gd,
                           const std::vector<Tile> &ordered) {
    if (b->d_tiles) cudaFree(b->d_tiles);
    b->d_tiles = nullptr;
    BCK(cudaMalloc(&b->d_tiles, sizeof(Tile) * std::max<size_t>(1, ordered.size())));
    BCK(cudaMemcpy(b->d_grids, gd.data(), sizeof(GridDesc) * gd.size(), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->d_tiles, ordered.data(), sizeof(Tile) * ordered.size(),
                   cudaMemcpyHostToDevice));
    b->ntiles = (int)ordered.size();
    b->built_a15f.clear();
    b->built_rounding.clear();
    for (const lbm_grid *g : b->grids) {
        b->built_a15f.push_back(g->a15f);
        b->built_rounding.push_back(g->rounding);
    }
    drop_graph(b);
    return LBM_OK;
}

// (Re)builds the device grid table and the tile work-list.
static int build_worklist(lbm_batch *b) {
    std::vector<GridDesc> gd(b->grids.size());
    std::vector<Tile> tiles;
    b->paired = 0;
    // Flow schedule: the kernel for the grids' kinds and the warps it keeps
    // resident, which set each grid's tile height below.
    FlowKernel fk = nullptr;
    int flow_bps = 1;
    long long flow_warps = 0;
    if (b->schedule == LBM_SCHEDULE_FLOW) {
        std::vector<int> kinds;
        for (const lbm_grid *g : b->grids)
            kinds.push_back(kind_code(g->storage, batch_vec(b, g), g->rounding ? 1 : 0,
                                      g->a15f ? 1 : 0));
        fk = flow_kernel_for(kinds, b->walk16);
        BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&flow_bps, (const void *)fk,
                                                          32 * kBatchWarps, 0));
        if (flow_bps < 1) return bfail(LBM_ECUDA, "flow kernel cannot be resident");
        const int per = b->blocks_per_sm > 0 ? std::min(b->blocks_per_sm, flow_bps) : flow_bps;
        flow_warps = (long long)per * b->sms * kBatchWarps;
    }
    // Lockstep, default configuration: every warp walks its tiles one after
    // another within a step, so a batch with fewer tiles than about the
    // resident warps (16 per SM in the specialised kernels) spends each step
    // on a whole walk with warps idle.  Such a batch gets shorter tiles, down
    // to 2 rows, as many as one wave holds.  Batches of at least 3/4 of a
    // wave of tiles keep the configured height.
    int lock_rows = b->rows;
    if (b->schedule == LBM_SCHEDULE_LOCKSTEP && b->fit_rows) {
        const int bps = b->blocks_per_sm > 0 ? b->blocks_per_sm : 4;
        const long long wave = (long long)bps * b->sms * kBatchWarps;
        auto tiles_at = [&](int r) {
            long long t = 0;
            for (const lbm_grid *g : b->grids) {
                const int w = 32 * batch_vec(b, g);
                t += (long long)((g->nx + w - 1) / w) * ((g->ny - 2 * g->slab + r - 1) / r);
            }
            return t;
        };
        if (4 * tiles_at(lock_rows) < 3 * wave)
            while (lock_rows > 2 && tiles_at(lock_rows - 1) <= wave) --lock_rows;
    }
    b->lock_rows = lock_rows;
    for (size_t k = 0; k < b->grids.size(); ++k) {
        lbm_grid *g = b->grids[k];
        GridDesc &d = gd[k];
        d.buf[0] = g->buf[0];
        d.buf[1] = g->buf[1];
        d.a15f = g->a15f;
        d.P = g->P;
        d.nx = g->nx;
        d.ny = g->ny;
        int v = batch_vec(b, g);
        d.kind = kind_code(g->storage, v, g->rounding ? 1 : 0, g->a15f ? 1 : 0);
        d.pad = 0;
        d.c = g->coef;
        int w = 32 * v;
        // Flow schedule: a grid's step takes at least one tile walk, so a grid
        // with fewer tiles than its share of the resident warps (the warps
        // split evenly between the grids) uses tiles a quarter as tall: four
        // times the tiles, each walk a quarter as long.
        int rows = lock_rows;
        if (b->schedule == LBM_SCHEDULE_FLOW) {
            const long long tiles_tall =
                (long long)((g->nx + w - 1) / w) * ((g->ny - 2 * g->slab + b->rows - 1) / b->rows);
            if (tiles_tall * (long long)b->grids.size() < flow_warps) rows = std::max(1, b->rows / 4);
        }
        // Rows computed: all of them, or a slab's own rows between its ghosts.
        const int ylo = g->slab, yhi = g->ny - g->slab, nyc = yhi - ylo;
        d.tile0 = (int)tiles.size();
        d.nstrips = (g->nx + w - 1) / w;
        d.nsegs = (nyc + rows - 1) / rows;
        d.ntile = d.nstrips * d.nsegs;
        // A step reads two rows and two columns beyond its tile: the next
        // segment or strip over suffices unless one of them is a single row
        // or column wide (the last one of a grid can be).
        const int last_rows = nyc - (d.nsegs - 1) * rows;
        const int last_cols = g->nx - (d.nstrips - 1) * w;
        d.dseg = (rows >= 2 && last_rows >= 2) ? 1 : 2;
        d.dstrip = last_cols >= 2 ? 1 : 2;
        // Neighbouring segments walk in opposite directions, so the rows they
        // share are read by both at about the same time (from L2 the second time).
        for (int y0 = ylo, seg = 0; y0 < yhi; y0 += rows, ++seg)
            for (int x0 = 0; x0 < g->nx; x0 += w)
                tiles.push_back(Tile{(int)k, x0, y0, std::min(yhi, y0 + rows),
                                     (seg & 1) ? -1 : 1});
    }
    if (b->schedule == LBM_SCHEDULE_FLOW) {
        // One launch over every grid, tiles grid by grid in their order.
        b->groups.clear();
        lbm_batch::Group gr;
        gr.begin = 0;
        gr.count = (int)tiles.size();
        gr.kernel = nullptr;
        gr.fkernel = fk;
        gr.max_blocks_per_sm = flow_bps;
        b->groups.push_back(gr);
        if (tiles.size() > b->prog_cap) {
            cudaFree(b->d_prog);
            b->d_prog = nullptr;
            BCK(cudaMalloc(&b->d_prog, sizeof(int) * tiles.size()));
            b->prog_cap = tiles.size();
        }
        if (!b->d_ctl)
            BCK(cudaMalloc(&b->d_ctl, sizeof(unsigned long long) * kFlowCtlWords *
                                          b->grids.size()));
        return upload_worklist(b, gd, tiles);
    }
    // Kind groups.  A kind with a specialised kernel runs in its own launch
    // when its grids move at least kOwnLaunchBytes per step (about 10 us of
    // HBM time, so the launch's fixed costs and its barrier stay small); all
    // other tiles share one launch of the general kernel, where small grids of
    // any kind overlap.  A batch of one kind is one group.
    constexpr double kOwnLaunchBytes = 64.0 * 1024 * 1024;
    std::vector<double> bytes(kKindCodes, 0.0);
    std::vector<int> count(kKindCodes, 0);
    for (size_t k = 0; k < b->grids.size(); ++k) {
        const lbm_grid *g = b->grids[k];
        bytes[gd[k].kind] += (double)g->nx * (g->ny - 2 * g->slab) *
                             ((g->storage == ST_F32 ? 72.0 : 36.0) + (g->a15f ? 4.0 : 0.0));
    }
    for (const Tile &t : tiles) count[gd[t.grid].kind]++;
    int kinds_present = 0;
    for (int kd = 0; kd < kKindCodes; ++kd) kinds_present += count[kd] > 0;
    std::vector<int> own, rest;
    for (int kd = 0; kd < kKindCodes; ++kd) {
        if (!count[kd]) continue;
        BatchKernel kk = kernel_for({kd}, b->walk16);
        if (kk != (BatchKernel)k_batch && (kinds_present == 1 || bytes[kd] >= kOwnLaunchBytes))
            own.push_back(kd);
        else
            rest.push_back(kd);
    }
    std::vector<Tile> ordered;
    ordered.reserve(tiles.size());
    b->groups.clear();
    // A group of one 8-site 16-bit kind (automatic walk) pairs the tiles of
    // its grids at most kSplitCols wide: consecutive segments share one warp,
    // a half-warp each (the split walk), where a single walk leaves half of
    // the lanes or more idle.  An odd one out stays single.  The kernel
    // instance with the split walk runs the whole-warp walk a few per cent
    // slower (its register allocation), and pairing the narrow last strip of
    // a wider grid measured no faster, so a group pairs only whole narrow
    // grids, and only when their tiles are at least kSplitMinShare of its
    // tiles.
    auto add_group = [&](const std::vector<int> &kinds_in) -> int {
        lbm_batch::Group gr;
        gr.begin = (int)ordered.size();
        auto in_group = [&](const Tile &t) {
            return std::find(kinds_in.begin(), kinds_in.end(), gd[t.grid].kind) != kinds_in.end();
        };
        auto narrow = [&](const Tile &t) { return gd[t.grid].nx <= kSplitCols; };
        bool split = kinds_in.size() == 1 && kind_splits(kinds_in[0]) &&
                     b->walk16 == LBM_WALK16_AUTO;
        if (split) {
            long long n_all = 0, n_narrow = 0;
            for (const Tile &t : tiles)
                if (in_group(t)) {
                    ++n_all;
                    n_narrow += narrow(t);
                }
            split = n_narrow > 0 && (double)n_narrow >= kSplitMinShare * (double)n_all;
        }
        const int paired0 = b->paired;
        std::vector<int> pending(b->grids.size(), -1);
        for (const Tile &t : tiles) {
            if (!in_group(t)) continue;
            if (split && narrow(t)) {
                int &p = pending[t.grid];
                if (p >= 0) {
                    Tile &a = ordered[p];
                    a.y0b = t.y0;
                    a.y1b = t.y1;
                    a.dirb = t.dir;
                    p = -1;
                    ++b->paired;
                    continue;
                }
                p = (int)ordered.size();
            }
            ordered.push_back(t);
        }
        // The end of each step: the warps that take the last tiles of a step
        // set its length, and the others wait at the barrier.  A group of more
        // than two waves of tiles splits its last wave's tiles in two (8 rows
        // each at the default height), halving that tail for one extra pulled
        // row pair per split tile.  Measured: the nine 2048^2 FP16-delta grids
        // 168.1k -> 170.2k MLUPS (stochastic rounding 165.0k -> 168.0k), the
        // 512-grid batch FP16-delta 158.6k -> 159.4k, FP32 sweep 93.4k ->
        // 93.8k; quarters, or halves over the last two waves, gained less.
        {
            const int bps = b->blocks_per_sm > 0 ? b->blocks_per_sm : 4;
            const long long wave = (long long)bps * b->sms * kBatchWarps;
            const long long n = (long long)ordered.size() - gr.begin;
            if (n > 2 * wave) {
                std::vector<Tile> tail(ordered.end() - wave, ordered.end());
                ordered.resize(ordered.size() - wave);
                for (const Tile &t : tail) {
                    if (t.y1b > t.y0b || t.y1 - t.y0 < 2) {
                        ordered.push_back(t);
                        continue;
                    }
                    const int mid = t.y0 + (t.y1 - t.y0) / 2;
                    ordered.push_back(Tile{t.grid, t.x0, t.y0, mid, 1});
                    ordered.push_back(Tile{t.grid, t.x0, mid, t.y1, -1});
                }
            }
        }
        gr.count = (int)ordered.size() - gr.begin;
        gr.kernel = kernel_for(kinds_in, b->walk16, b->paired > paired0);
        BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&gr.max_blocks_per_sm,
                                                          (const void *)gr.kernel,
                                                          32 * kBatchWarps, 0));
        if (gr.max_blocks_per_sm < 1) return bfail(LBM_ECUDA, "batch kernel cannot be resident");
        b->groups.push_back(gr);
        return LBM_OK;
    };
    for (int kd : own) {
        int rc = add_group({kd});
        if (rc != LBM_OK) return rc;
    }
    if (!rest.empty()) {
        int rc = add_group(rest);
        if (rc != LBM_OK) return rc;
    }
    return upload_worklist(b, gd, ordered);
}

extern "C" int lbm_batch_destroy(lbm_batch_t b) {
    if (!b) return LBM_OK;
    if (b->stream || b->d_grids) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    cudaFree(b->d_grids);
    cudaFree(b->d_tiles);
    cudaFree(b->d_limit);
    cudaFree(b->d_parity);
    cudaFree(b->d_t0);
    cudaFree(b->d_bar);
    cudaFree(b->d_status);
    cudaFree(b->d_ctl);
    cudaFree(b->d_prog);
    cudaFree(b->d_nwork);
    if (b->h_nwork) cudaFreeHost(b->h_nwork);
    if (b->h_limit) cudaFreeHost(b->h_limit);
    if (b->h_parity) cudaFreeHost(b->h_parity);
    if (b->h_t0) cudaFreeHost(b->h_t0);
    if (b->h_status) cudaFreeHost(b->h_status);
    if (b->copied) cudaEventDestroy(b->copied);
    for (cudaEvent_t ev : b->xev) cudaEventDestroy(ev);
    if (b->done) cudaEventDestroy(b->done);
    delete b;
    return LBM_OK;
}

extern "C" int lbm_batch_create(const lbm_t *grids, int n, lbm_batch_t *out) {
    if (!out || !grids || n < 1) return bfail(LBM_EINVAL, "lbm_batch_create: bad argument");
    *out = nullptr;
    for (int k = 0; k < n; ++k) {
        if (!grids[k]) return bfail(LBM_EINVAL, "lbm_batch_create: NULL grid");
        if (grids[k]->drive)
            return bfail(LBM_EINVAL, "lbm_batch_create: driven grids are not batched");
        if (grids[k]->grad != LBM_GRAD_CENTRAL)
            return bfail(LBM_EINVAL, "lbm_batch_create: the batch kernels use the central "
                                     "difference (lbm_set_gradient)");
    }
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return bfail(LBM_ENOMEM, "lbm_batch_create: host allocation failed");
    b->grids.assign(grids, grids + n);
    b->stream = grids[0]->stream;
    b->device = grids[0]->device;
    for (int k = 0; k < n; ++k)
        if (grids[k]->device != b->device) {
            delete b;
            return bfail(LBM_EINVAL, "lbm_batch_create: grids on different devices");
        }
    // One attribute (a full cudaGetDeviceProperties is slow, and servers
    // re-create batches often).
    cudaError_t e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_grids, sizeof(GridDesc) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_limit, sizeof(long long) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_parity, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_t0, sizeof(uint32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_bar, sizeof(unsigned) * kBarWords);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_limit, sizeof(long long) * n);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_parity, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_t0, sizeof(uint32_t) * n);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_nwork, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_nwork, sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int));
    if (e != cudaSuccess) {
        int rc = bcuda(e, "lbm_batch_create");
        lbm_batch_destroy(b);
        return rc;
    }
    int rc = build_worklist(b);
    if (rc != LBM_OK) {
        lbm_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LBM_OK;
}

static int grid_blocks(const lbm_batch *b, const lbm_batch::Group &g) {
    int per = b->blocks_per_sm > 0 ? std::min(b->blocks_per_sm, g.max_blocks_per_sm)
                                   : g.max_blocks_per_sm;
    return per * b->sms;
}

// Queues: copy per-call arrays, reset barrier and status, cooperative launch.
static cudaError_t enqueue(lbm_batch *b, long long n, cudaStream_t st) {
    int ng = (int)b->grids.size();
    cudaError_t e = cudaMemcpyAsync(b->d_limit, b->h_limit, sizeof(long long) * ng,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_parity, b->h_parity, sizeof(int) * ng, cudaMemcpyHostToDevice,
                            st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_t0, b->h_t0, sizeof(uint32_t) * ng, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const GridDesc *grids = b->d_grids;
    const long long *lim = b->d_limit;
    const int *par = b->d_parity;
    const uint32_t *t0 = b->d_t0;
    unsigned *bar = b->d_bar;
    int *status = b->d_status;
    unsigned long long to = b->timeout_ns;
    if (b->schedule == LBM_SCHEDULE_FLOW) {
        e = cudaMemcpyAsync(b->d_nwork, b->h_nwork, sizeof(int), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(b->d_ctl, 0,
                                sizeof(unsigned long long) * kFlowCtlWords * ng, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_prog, 0, sizeof(int) * b->ntiles, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned) * kBarWords, st);
        if (e != cudaSuccess) return e;
        b->groups[0].fkernel<<<grid_blocks(b, b->groups[0]), 32 * kBatchWarps, 0, st>>>(
            grids, ng, b->d_tiles, lim, par, t0, b->d_ctl, b->d_prog, bar, b->d_nwork, status,
            to);
        return cudaGetLastError();
    }
    // The groups hold disjoint grids: each launch advances its grids by all n
    // steps.  Barrier words and tile counters start at zero for every launch.
    for (const lbm_batch::Group &gr : b->groups) {
        e = cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned) * kBarWords, st);
        if (e != cudaSuccess) return e;
        const Tile *tiles = b->d_tiles + gr.begin;
        int ntiles = gr.count;
        void *args[] = {(void *)&grids, (void *)&tiles, (void *)&ntiles, (void *)&lim,
                        (void *)&par,   (void *)&t0,    (void *)&n,      (void *)&bar,
                        (void *)&status, (void *)&to};
        e = cudaLaunchCooperativeKernel((const void *)gr.kernel, dim3(grid_blocks(b, gr)),
                                        dim3(32 * kBatchWarps), args, 0, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static int run_batch(lbm_batch *b, long long n, const long long *limits, bool advance) {
    int ng = (int)b->grids.size();
    // The previous call's copies must have read the pinned arrays first.
    BCK(cudaEventSynchronize(b->copied));
    int nwork = 0;
    for (int k = 0; k < ng; ++k) {
        long long lim = limits ? std::max(0LL, std::min(n, limits[k])) : n;
        b->h_limit[k] = lim;
        b->h_parity[k] = b->grids[k]->cur;
        b->h_t0[k] = (uint32_t)b->grids[k]->t;
        nwork += lim > 0;
    }
    *b->h_nwork = nwork;
    // Work already queued on the members' own streams (an lbm_init, a step
    // call) runs before the batch's launches.
    int nxs = 0;
    for (const lbm_grid *g : b->grids) {
        cudaStream_t s = g->stream;
        if (s == b->stream || std::find(b->xs.begin(), b->xs.begin() + nxs, s) != b->xs.begin() + nxs)
            continue;
        if (nxs == (int)b->xs.size()) {
            cudaEvent_t ev = nullptr;
            BCK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            b->xev.push_back(ev);
            b->xs.push_back(s);
        }
        b->xs[nxs] = s;
        BCK(cudaEventRecord(b->xev[nxs], s));
        BCK(cudaStreamWaitEvent(b->stream, b->xev[nxs], 0));
        ++nxs;
    }
    cudaError_t e = cudaSuccess;
    const bool want_graph = b->launch_mode == LBM_LAUNCH_GRAPH ||
                            (b->launch_mode == LBM_LAUNCH_AUTO && !b->capture_failed);
    bool graphed = false;
    if (want_graph) {
        if (b->graph_n != n) {
            drop_graph(b);
            cudaStream_t cs;
            BCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e1 = enqueue(b, n, cs);
                cudaError_t e2 = cudaStreamEndCapture(cs, &g);
                e = e1 != cudaSuccess ? e1 : e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            if (e != cudaSuccess) {
                cudaGetLastError();
                drop_graph(b);
                if (b->launch_mode == LBM_LAUNCH_GRAPH)
                    return bcuda(e, "lbm_batch_step: capturing the persistent launch in a CUDA graph");
                // AUTO: recorded (lbm_batch_get_launch) and never retried.
                b->capture_failed = true;
            } else {
                b->graph_n = n;
            }
        }
        if (b->graph) {
            e = cudaGraphLaunch(b->graph, b->stream);
            graphed = true;
        }
    }
    if (!graphed) e = enqueue(b, n, b->stream);
    if (e != cudaSuccess) return bcuda(e, "lbm_batch_step launch");
    b->last_launch = graphed ? LBM_LAUNCH_GRAPH : LBM_LAUNCH_DIRECT;
    BCK(cudaEventRecord(b->copied, b->stream));
    if (nxs) {
        // Later work on those streams (lbm_moments, lbm_destroy, a step)
        // waits for the batch's.
        BCK(cudaEventRecord(b->done, b->stream));
        for (int k = 0; k < nxs; ++k) BCK(cudaStreamWaitEvent(b->xs[k], b->done, 0));
    }
    if (advance) {
        for (int k = 0; k < ng; ++k) {
            long long s = b->h_limit[k];
            b->grids[k]->t += s;
            if (s & 1) b->grids[k]->cur ^= 1;
        }
    }
    return LBM_OK;
}

extern "C" int lbm_batch_step(lbm_batch_t b, long long n, const long long *limits) {
    if (!b || n < 0) return bfail(LBM_EINVAL, "lbm_batch_step: bad argument");
    if (b->schedule == LBM_SCHEDULE_FLOW && n > 0x7fffffffLL)
        return bfail(LBM_EINVAL, "lbm_batch_step: flow schedule takes at most 2^31 - 1 steps a call");
    if (n == 0) return LBM_OK;
    bool stale = false;
    for (size_t k = 0; k < b->grids.size(); ++k) {
        const lbm_grid *g = b->grids[k];
        if (g->drive) return bfail(LBM_EINVAL, "lbm_batch_step: a grid has a drive");
        if (g->grad != LBM_GRAD_CENTRAL)
            return bfail(LBM_EINVAL, "lbm_batch_step: a grid uses the forward difference");
        stale = stale || g->a15f != b->built_a15f[k] || g->rounding != b->built_rounding[k];
    }
    if (stale) {
        // A grid's c2 field or rounding changed since the work-list was built.
        BCK(cudaStreamSynchronize(b->stream));
        int rc = build_worklist(b);
        if (rc != LBM_OK) return rc;
    }
    return run_batch(b, n, limits, true);
}

cudaError_t batch_queue_status(lbm_batch *b, cudaStream_t st) {
    return cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
}

int batch_status(const lbm_batch *b) { return *b->h_status; }

extern "C" int lbm_batch_sync(lbm_batch_t b) {
    if (!b) return bfail(LBM_EINVAL, "lbm_batch_sync: NULL batch");
    BCK(cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                        b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    if (*b->h_status != 0)
        return bfail(*b->h_status, "lbm_batch_sync: a barrier wait in the batch kernel ran out");
    return LBM_OK;
}

extern "C" int lbm_batch_set_config(lbm_batch_t b, int rows, int blocks_per_sm) {
    if (!b || rows < 1 || rows > 4096 || blocks_per_sm < 0)
        return bfail(LBM_EINVAL, "lbm_batch_set_config: bad argument");
    BCK(cudaStreamSynchronize(b->stream));
    b->blocks_per_sm = blocks_per_sm;
    if (rows != b->rows || b->fit_rows) {
        b->rows = rows;
        b->fit_rows = false;
        return build_worklist(b);
    }
    drop_graph(b);
    return LBM_OK;
}

extern "C" int lbm_batch_set_walk16(lbm_batch_t b, int walk) {
    if (!b || walk < LBM_WALK16_AUTO || walk > LBM_WALK16_V4_PF2)
        return bfail(LBM_EINVAL, "lbm_batch_set_walk16: unknown walk");
    BCK(cudaStreamSynchronize(b->stream));
    if (walk == b->walk16) return LBM_OK;
    b->walk16 = walk;
    return build_worklist(b);
}

extern "C" int lbm_batch_get_walk16(lbm_batch_t b, int *walk) {
    if (!b || !walk) return bfail(LBM_EINVAL, "lbm_batch_get_walk16: bad argument");
    *walk = b->walk16;
    return LBM_OK;
}

extern "C" int lbm_batch_get_groups(lbm_batch_t b, int *groups) {
    if (!b || !groups) return bfail(LBM_EINVAL, "lbm_batch_get_groups: bad argument");
    *groups = (int)b->groups.size();
    return LBM_OK;
}

extern "C" int lbm_batch_set_timeout_us(lbm_batch_t b, long long us) {
    if (!b || us < 1) return bfail(LBM_EINVAL, "lbm_batch_set_timeout_us: bad argument");
    b->timeout_ns = (unsigned long long)us * 1000ULL;
    drop_graph(b);
    return LBM_OK;
}

// Times one-step dry runs (the state is not advanced: every grid writes its
// other buffer) for several tile heights and, when the batch holds 16-bit
// grids, the 16-bit walks, each at its full occupancy; keeps the fastest.
// A one-step launch does the same per-step work as a step inside a longer
// launch (the barriers between steps cost microseconds per millisecond step).
// Times dry one-step runs of every (walk, tile height) candidate with the
// events e0/e1 and leaves the fastest in *rows / *walk.
static int tune_candidates(lbm_batch *b, cudaEvent_t e0, cudaEvent_t e1, int *rows,
                           int *walk_out) {
    float best = 1e30f;
    const int rowss[] = {8, 12, 16, 24, 32};
    std::vector<std::vector<BatchKernel>> seen;
    for (int walk = LBM_WALK16_AUTO; walk <= LBM_WALK16_V4_PF2; ++walk) {
        int rc = lbm_batch_set_walk16(b, walk);
        if (rc != LBM_OK) return rc;
        std::vector<BatchKernel> ks;
        for (const auto &gr : b->groups) ks.push_back(gr.kernel);
        if (std::find(seen.begin(), seen.end(), ks) != seen.end()) continue;  // same kernels
        seen.push_back(ks);
        for (int r : rowss) {
            rc = lbm_batch_set_config(b, r, 0);
            if (rc != LBM_OK) return rc;
            rc = run_batch(b, 1, nullptr, false);  // warm-up (and graph build)
            if (rc != LBM_OK) return rc;
            BCK(cudaEventRecord(e0, b->stream));
            for (int k = 0; k < 4 && rc == LBM_OK; ++k) rc = run_batch(b, 1, nullptr, false);
            if (rc != LBM_OK) return rc;
            BCK(cudaEventRecord(e1, b->stream));
            BCK(cudaEventSynchronize(e1));
            float ms = 0.f;
            BCK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                *rows = r;
                *walk_out = walk;
            }
        }
    }
    return LBM_OK;
}

extern "C" int lbm_batch_tune(lbm_batch_t b) {
    if (!b) return bfail(LBM_EINVAL, "lbm_batch_tune: NULL batch");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCK(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return bcuda(e, "cudaEventCreate");
    }
    const int rows0 = b->rows, walk0 = b->walk16, bps0 = b->blocks_per_sm;
    const bool fit0 = b->fit_rows;
    int best_rows = rows0, best_walk = walk0;
    int rc = tune_candidates(b, e0, e1, &best_rows, &best_walk);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LBM_OK) {
        // The configuration in force before the call is put back.
        lbm_batch_set_walk16(b, walk0);
        lbm_batch_set_config(b, rows0, bps0);
        if (fit0) {
            b->fit_rows = true;
            build_worklist(b);
        }
        return rc;
    }
    rc = lbm_batch_set_walk16(b, best_walk);
    return rc != LBM_OK ? rc : lbm_batch_set_config(b, best_rows, 0);
}

extern "C" int lbm_batch_set_schedule(lbm_batch_t b, int schedule) {
    if (!b || schedule < LBM_SCHEDULE_LOCKSTEP || schedule > LBM_SCHEDULE_FLOW)
        return bfail(LBM_EINVAL, "lbm_batch_set_schedule: unknown schedule");
    BCK(cudaStreamSynchronize(b->stream));
    if (schedule == b->schedule) return LBM_OK;
    b->schedule = schedule;
    return build_worklist(b);
}

extern "C" int lbm_batch_get_schedule(lbm_batch_t b, int *schedule) {
    if (!b || !schedule) return bfail(LBM_EINVAL, "lbm_batch_get_schedule: bad argument");
    *schedule = b->schedule;
    return LBM_OK;
}

extern "C" int lbm_batch_set_launch(lbm_batch_t b, int mode) {
    if (!b || mode < LBM_LAUNCH_AUTO || mode > LBM_LAUNCH_DIRECT)
        return bfail(LBM_EINVAL, "lbm_batch_set_launch: unknown mode");
    BCK(cudaStreamSynchronize(b->stream));
    b->launch_mode = mode;
    b->capture_failed = false;
    drop_graph(b);
    return LBM_OK;
}

extern "C" int lbm_batch_get_launch(lbm_batch_t b, int *mode, int *last, int *capture_failed) {
    if (!b) return bfail(LBM_EINVAL, "lbm_batch_get_launch: NULL batch");
    if (mode) *mode = b->launch_mode;
    if (last) *last = b->last_launch;
    if (capture_failed) *capture_failed = b->capture_failed ? 1 : 0;
    return LBM_OK;
}

extern "C" int lbm_batch_get_tiles(lbm_batch_t b, int *tiles, int *paired) {
    if (!b) return bfail(LBM_EINVAL, "lbm_batch_get_tiles: NULL batch");
    if (tiles) *tiles = b->ntiles;
    if (paired) *paired = b->paired;
    return LBM_OK;
}

extern "C" int lbm_batch_get_config(lbm_batch_t b, int *rows, int *blocks_per_sm,
                                    int *specialised) {
    if (!b) return bfail(LBM_EINVAL, "lbm_batch_get_config: NULL batch");
    if (rows) *rows = b->schedule == LBM_SCHEDULE_LOCKSTEP ? b->lock_rows : b->rows;
    if (blocks_per_sm)
        *blocks_per_sm = b->groups.empty() ? 0 : grid_blocks(b, b->groups[0]) / b->sms;
    if (specialised) {
        *specialised = 1;
        for (const auto &gr : b->groups)
            if (gr.kernel == (BatchKernel)k_batch || gr.fkernel == (FlowKernel)k_flow)
                *specialised = 0;
    }
    return LBM_OK;
}
