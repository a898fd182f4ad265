// Batched form: many uneven grids (any size, tau, c2 and storage) advanced by
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

using namespace vss;

namespace {

struct GridDesc {
    void *buf[2];
    const float *a15f;  // 1.5 alpha per site for a grid with a c2 field, else NULL
    size_t P;
    int nx, ny;
    int kind;  // kind_code(storage, vec, stochastic rounding)
    int pad;
    Coef c;
};

struct Tile {
    int grid, x0, y0, y1, dir;
};

// A grid's walk in the batch kernels: storage kind, sites per lane (1, 4 or
// 8), stochastic rounding, and a per-site c2 field.
constexpr int kind_code(int storage, int vec, int sr, int va = 0) {
    return storage * 64 + vec + 16 * sr + 32 * va;
}
constexpr int kKindCodes = 3 * 64;

constexpr int kBatchWarps = 4;  // warps per block of the persistent kernel

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Barrier and scheduling words, each on its own 128-byte line: the arrival
// count, the generation the waiting blocks poll, and the two tile counters
// (the counters' atomics must not queue behind the polling).
constexpr int kBarGen = 32;     // generation (word offset)
constexpr int kCtr = 64;        // tile counter of even steps; odd steps at kCtr + 32
constexpr int kBarWords = 128;  // words allocated

// Grid-wide barrier over all blocks of a cooperative launch.  bar[0] counts
// arrivals, bar[kBarGen] is the generation.  Waiting blocks poll with a
// sleep that doubles from 64 ns to 1 us, and look at the status word and the
// clock every 16 polls.  Returns false if the wait ran out or another block
// reported an error.
__device__ bool grid_barrier(unsigned *bar, int *status, unsigned long long timeout_ns) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *vgen = bar + kBarGen;
        unsigned gen = *vgen;
        __threadfence();
        unsigned prev = atomicAdd(bar, 1u);
        if (prev == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + kBarGen, 1u);
        } else {
            unsigned long long t0 = global_ns();
            unsigned ns = 64;
            for (unsigned it = 0; *vgen == gen; ++it) {
                if ((it & 15u) == 15u) {
                    if (*(volatile int *)status != 0) {
                        ok = 0;
                        break;
                    }
                    if (global_ns() - t0 > timeout_ns) {
                        atomicCAS(status, 0, LBM_ETIMEOUT);
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(ns);
                if (ns < 1024u) ns *= 2u;
            }
        }
        __threadfence();
        if (*(volatile int *)status != 0) ok = 0;
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

// Dynamic tile scheduling: within a time step, warps take the next tile
// index from a counter (one per step parity; the counter of step k is reset
// during step k+1, and the barrier at the end of k+1 orders that reset before
// step k+2 uses it again).  Uneven tiles then balance across warps.
__device__ __forceinline__ unsigned *step_counter(unsigned *bar, long long k) {
    return bar + kCtr + 32 * (int)(k & 1);
}

__device__ __forceinline__ int next_tile(unsigned *ctr) {
    unsigned v = 0;
    if ((threadIdx.x & 31) == 0) v = atomicAdd(ctr, 1u);
    return (int)__shfl_sync(FULL, v, 0);
}

__device__ __forceinline__ void reset_counter(unsigned *bar, long long k) {
    if (k >= 1 && blockIdx.x == 0 && threadIdx.x == 0) *step_counter(bar, k - 1) = 0u;
}

template <int S, int V, bool PF = false, int RND = 0, int VA = 0>
__device__ __noinline__ void do_tile(const GridDesc &g, int par, const Tile &t, uint32_t step) {
    Walker<S, V, LD_CG, RND, VA> w(g.buf[par], g.buf[par ^ 1], g.nx, g.ny, g.P, t.x0);
    if constexpr (VA) w.a15f = g.a15f;
    if constexpr (RND) w.rstep = step;
    if constexpr (PF)
        w.run_prefetch(t.y0, t.y1, t.dir, g.c);
    else
        w.run(t.y0, t.y1, t.dir, g.c);
}

__global__ void __launch_bounds__(32 * kBatchWarps, 3)
    k_batch(const GridDesc *__restrict__ grids, const Tile *__restrict__ tiles, int ntiles,
            const long long *__restrict__ limit, const int *__restrict__ parity0,
            const uint32_t *__restrict__ t0, long long nsteps, unsigned *bar, int *status,
            unsigned long long timeout_ns) {
    for (long long k = 0; k < nsteps; ++k) {
        reset_counter(bar, k);
        unsigned *ctr = step_counter(bar, k);
        for (int ti = next_tile(ctr); ti < ntiles; ti = next_tile(ctr)) {
            const Tile t = tiles[ti];
            if (k >= limit[t.grid]) continue;
            const GridDesc &g = grids[t.grid];
            const int par = (parity0[t.grid] + (int)(k & 1)) & 1;
            const uint32_t step = t0[t.grid] + (uint32_t)k;
            switch (g.kind) {
                case kind_code(ST_F32, 4, 0):
                    do_tile<ST_F32, 4>(g, par, t, step);
                    break;
                case kind_code(ST_F32, 1, 0):
                    do_tile<ST_F32, 1>(g, par, t, step);
                    break;
                case kind_code(ST_F16, 8, 0):
                    do_tile<ST_F16, 8>(g, par, t, step);
                    break;
                case kind_code(ST_F16, 4, 0):
                    do_tile<ST_F16, 4, true>(g, par, t, step);
                    break;
                case kind_code(ST_F16, 1, 0):
                    do_tile<ST_F16, 1>(g, par, t, step);
                    break;
                case kind_code(ST_BF16, 8, 0):
                    do_tile<ST_BF16, 8>(g, par, t, step);
                    break;
                case kind_code(ST_BF16, 4, 0):
                    do_tile<ST_BF16, 4, true>(g, par, t, step);
                    break;
                case kind_code(ST_BF16, 1, 0):
                    do_tile<ST_BF16, 1>(g, par, t, step);
                    break;
                case kind_code(ST_F16, 8, 1):
                    do_tile<ST_F16, 8, false, 1>(g, par, t, step);
                    break;
                case kind_code(ST_F16, 4, 1):
                    do_tile<ST_F16, 4, true, 1>(g, par, t, step);
                    break;
                case kind_code(ST_F16, 1, 1):
                    do_tile<ST_F16, 1, false, 1>(g, par, t, step);
                    break;
                case kind_code(ST_BF16, 8, 1):
                    do_tile<ST_BF16, 8, false, 1>(g, par, t, step);
                    break;
                case kind_code(ST_BF16, 4, 1):
                    do_tile<ST_BF16, 4, true, 1>(g, par, t, step);
                    break;
                case kind_code(ST_BF16, 1, 1):
                    do_tile<ST_BF16, 1, false, 1>(g, par, t, step);
                    break;
                case kind_code(ST_F32, 4, 0, 1):
                    do_tile<ST_F32, 4, false, 0, 1>(g, par, t, step);
                    break;
                case kind_code(ST_F32, 1, 0, 1):
                    do_tile<ST_F32, 1, false, 0, 1>(g, par, t, step);
                    break;
                case kind_code(ST_F16, 4, 0, 1):
                    do_tile<ST_F16, 4, true, 0, 1>(g, par, t, step);
                    break;
                case kind_code(ST_F16, 1, 0, 1):
                    do_tile<ST_F16, 1, false, 0, 1>(g, par, t, step);
                    break;
                case kind_code(ST_BF16, 4, 0, 1):
                    do_tile<ST_BF16, 4, true, 0, 1>(g, par, t, step);
                    break;
                case kind_code(ST_BF16, 1, 0, 1):
                    do_tile<ST_BF16, 1, false, 0, 1>(g, par, t, step);
                    break;
                default:
                    break;
            }
        }
        if (k + 1 < nsteps && !grid_barrier(bar, status, timeout_ns)) return;
    }
}

// Specialised persistent kernel for a batch whose grids all use one walk
// (storage, vec, rounding, rows of loads in flight PD = 0, 1 or 2): the walk is
// inlined, so the kernel keeps the single-grid kernel's register budget (128,
// 16 warps per SM; 170 and 12 warps per SM for the two-row prefetch) instead
// of paying for calls.  Same time-step loop and bounded barrier as k_batch.
template <int S, int V, int PD, int RND, int VA = 0>
__global__ void __launch_bounds__(32 * kBatchWarps, PD == 2 ? 3 : 4)
    k_batch_one(const GridDesc *__restrict__ grids, const Tile *__restrict__ tiles, int ntiles,
                const long long *__restrict__ limit, const int *__restrict__ parity0,
                const uint32_t *__restrict__ t0, long long nsteps, unsigned *bar, int *status,
                unsigned long long timeout_ns) {
    // Row buffers of the 8-site 16-bit walks: per warp a landing slot and a
    // stash of 9 x 32 16-byte vectors each (36 KiB per block).
    __shared__ uint4 rowbuf[(S != ST_F32 && V == 8) ? kBatchWarps : 1][2 * 9 * 32];
    (void)rowbuf;
    for (long long k = 0; k < nsteps; ++k) {
        reset_counter(bar, k);
        unsigned *ctr = step_counter(bar, k);
        for (int ti = next_tile(ctr); ti < ntiles; ti = next_tile(ctr)) {
            const Tile t = tiles[ti];
            if (k >= limit[t.grid]) continue;
            // Fields are read through a reference: a local copy indexed by the
            // run-time parity would live in local memory.
            const GridDesc &g = grids[t.grid];
            const int par = (parity0[t.grid] + (int)(k & 1)) & 1;
            const Coef c = g.c;
            Walker<S, V, LD_CG, RND, VA> w(g.buf[par], g.buf[par ^ 1], g.nx, g.ny, g.P, t.x0);
            if constexpr (VA) w.a15f = g.a15f;
            if constexpr (RND) w.rstep = t0[t.grid] + (uint32_t)k;
            if constexpr (S != ST_F32 && V == 8)
                w.run_async(t.y0, t.y1, t.dir, c, &rowbuf[threadIdx.x >> 5][0]);
            else if constexpr (PD == 2)
                w.run_prefetch2(t.y0, t.y1, t.dir, c);
            else if constexpr (PD == 1)
                w.run_prefetch(t.y0, t.y1, t.dir, c);
            else
                w.run(t.y0, t.y1, t.dir, c);
        }
        if (k + 1 < nsteps && !grid_barrier(bar, status, timeout_ns)) return;
    }
}

using BatchKernel = void (*)(const GridDesc *, const Tile *, int, const long long *, const int *,
                             const uint32_t *, long long, unsigned *, int *, unsigned long long);

// The kernel for a set of kinds: a specialised one when every grid has the
// same kind, else the general k_batch.  `walk16` picks the prefetch depth of
// the 16-bit vec 4 walks (LBM_WALK16_V4: one row, LBM_WALK16_V4_PF2: two).
BatchKernel kernel_for(const std::vector<int> &kinds, int walk16) {
    bool same = true;
    for (int k : kinds) same = same && k == kinds[0];
    if (!kinds.empty() && same) {
        const bool two = walk16 == LBM_WALK16_V4_PF2;
        switch (kinds[0]) {
            case kind_code(ST_F32, 4, 0):
                return k_batch_one<ST_F32, 4, 0, 0>;
            case kind_code(ST_F16, 8, 0):
                return k_batch_one<ST_F16, 8, 0, 0>;
            case kind_code(ST_BF16, 8, 0):
                return k_batch_one<ST_BF16, 8, 0, 0>;
            case kind_code(ST_F16, 8, 1):
                return k_batch_one<ST_F16, 8, 0, 1>;
            case kind_code(ST_BF16, 8, 1):
                return k_batch_one<ST_BF16, 8, 0, 1>;
            case kind_code(ST_F16, 4, 0):
                return two ? k_batch_one<ST_F16, 4, 2, 0> : k_batch_one<ST_F16, 4, 1, 0>;
            case kind_code(ST_BF16, 4, 0):
                return two ? k_batch_one<ST_BF16, 4, 2, 0> : k_batch_one<ST_BF16, 4, 1, 0>;
            case kind_code(ST_F16, 4, 1):
                return two ? k_batch_one<ST_F16, 4, 2, 1> : k_batch_one<ST_F16, 4, 1, 1>;
            case kind_code(ST_BF16, 4, 1):
                return two ? k_batch_one<ST_BF16, 4, 2, 1> : k_batch_one<ST_BF16, 4, 1, 1>;
            case kind_code(ST_F32, 4, 0, 1):
                return k_batch_one<ST_F32, 4, 0, 0, 1>;
            case kind_code(ST_F16, 4, 0, 1):
                return k_batch_one<ST_F16, 4, 1, 0, 1>;
            case kind_code(ST_BF16, 4, 0, 1):
                return k_batch_one<ST_BF16, 4, 1, 0, 1>;
            default:
                break;
        }
    }
    return k_batch;
}

}  // namespace

struct lbm_batch {
    std::vector<lbm_grid *> grids;
    // Per grid, the c2 field pointer and rounding mode the work-list was built
    // for (a change rebuilds it at the next step call).
    std::vector<const float *> built_a15f;
    std::vector<int> built_rounding;
    cudaStream_t stream = nullptr;
    int device = 0;
    int rows = 16;
    int blocks_per_sm = 0;  // 0: the occupancy limit
    // Kind groups: consecutive ranges of the tile list, each run by its own
    // persistent launch (a specialised k_batch_one, or k_batch for the rest),
    // one after the other on the batch's stream.
    struct Group {
        int begin = 0, count = 0;
        BatchKernel kernel = nullptr;
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
    // graph cache (one step count)
    cudaGraphExec_t graph = nullptr;
    long long graph_n = -1;
    bool use_graph = true;
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
// multiple of 4.  16-bit without a c2 field: 8 (128-bit loads, rows through
// shared memory) when nx is a multiple of 8 and the walk is LBM_WALK16_AUTO
// or LBM_WALK16_V8; else 4 (64-bit loads, one row prefetched in registers)
// when nx is a multiple of 4.  Any other nx: 1.  (Measured on GB300: 8 sites
// per lane run 15 % faster than 4 with nearest rounding and 10 % faster with
// stochastic rounding.)
static int batch_vec(const lbm_batch *b, const lbm_grid *g) {
    const bool eight = !g->a15f && (b->walk16 == LBM_WALK16_V8 || b->walk16 == LBM_WALK16_AUTO);
    if (g->storage != ST_F32 && eight && g->nx % 8 == 0) return 8;
    return g->nx % 4 == 0 ? 4 : 1;
}

// (Re)builds the device grid table and the tile work-list.
static int build_worklist(lbm_batch *b) {
    std::vector<GridDesc> gd(b->grids.size());
    std::vector<Tile> tiles;
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
        // Neighbouring segments walk in opposite directions, so the rows they
        // share are read by both at about the same time (from L2 the second time).
        for (int y0 = 0, seg = 0; y0 < g->ny; y0 += b->rows, ++seg)
            for (int x0 = 0; x0 < g->nx; x0 += w)
                tiles.push_back(Tile{(int)k, x0, y0, std::min(g->ny, y0 + b->rows),
                                     (seg & 1) ? -1 : 1});
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
        bytes[gd[k].kind] += (double)g->nx * g->ny *
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
    auto add_group = [&](const std::vector<int> &kinds_in) -> int {
        lbm_batch::Group gr;
        gr.begin = (int)ordered.size();
        for (const Tile &t : tiles) {
            int kd = gd[t.grid].kind;
            if (std::find(kinds_in.begin(), kinds_in.end(), kd) != kinds_in.end())
                ordered.push_back(t);
        }
        gr.count = (int)ordered.size() - gr.begin;
        gr.kernel = kernel_for(kinds_in, b->walk16);
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
    if (b->h_limit) cudaFreeHost(b->h_limit);
    if (b->h_parity) cudaFreeHost(b->h_parity);
    if (b->h_t0) cudaFreeHost(b->h_t0);
    if (b->h_status) cudaFreeHost(b->h_status);
    if (b->copied) cudaEventDestroy(b->copied);
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
    cudaError_t e = cudaSuccess;
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, b->device);
    if (e == cudaSuccess) b->sms = prop.multiProcessorCount;
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
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming);
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
    for (int k = 0; k < ng; ++k) {
        long long lim = limits ? std::max(0LL, std::min(n, limits[k])) : n;
        b->h_limit[k] = lim;
        b->h_parity[k] = b->grids[k]->cur;
        b->h_t0[k] = (uint32_t)b->grids[k]->t;
    }
    cudaError_t e = cudaSuccess;
    if (b->use_graph) {
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
                // Cooperative launches that cannot be captured run directly.
                cudaGetLastError();
                b->use_graph = false;
                drop_graph(b);
            } else {
                b->graph_n = n;
            }
        }
        if (b->use_graph) e = cudaGraphLaunch(b->graph, b->stream);
    }
    if (!b->use_graph) e = enqueue(b, n, b->stream);
    if (e != cudaSuccess) return bcuda(e, "lbm_batch_step launch");
    BCK(cudaEventRecord(b->copied, b->stream));
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
    if (n == 0) return LBM_OK;
    bool stale = false;
    for (size_t k = 0; k < b->grids.size(); ++k) {
        const lbm_grid *g = b->grids[k];
        if (g->drive) return bfail(LBM_EINVAL, "lbm_batch_step: a grid has a drive");
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
    if (rows != b->rows) {
        b->rows = rows;
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
    int best_rows = rows0, best_walk = walk0;
    int rc = tune_candidates(b, e0, e1, &best_rows, &best_walk);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LBM_OK) {
        // The configuration in force before the call is put back.
        lbm_batch_set_walk16(b, walk0);
        lbm_batch_set_config(b, rows0, bps0);
        return rc;
    }
    rc = lbm_batch_set_walk16(b, best_walk);
    return rc != LBM_OK ? rc : lbm_batch_set_config(b, best_rows, 0);
}

extern "C" int lbm_batch_get_config(lbm_batch_t b, int *rows, int *blocks_per_sm,
                                    int *specialised) {
    if (!b) return bfail(LBM_EINVAL, "lbm_batch_get_config: NULL batch");
    if (rows) *rows = b->rows;
    if (blocks_per_sm)
        *blocks_per_sm = b->groups.empty() ? 0 : grid_blocks(b, b->groups[0]) / b->sms;
    if (specialised) {
        *specialised = 1;
        for (const auto &gr : b->groups)
            if (gr.kernel == (BatchKernel)k_batch) *specialised = 0;
    }
    return LBM_OK;
}
