// Device side of the batched form: the grid descriptor and tile records,
// the bounded grid barrier, the per-step tile counters and the persistent
// batch kernels (the general k_batch and the specialised k_batch_one), plus
// the table that picks a kernel for a set of grid kinds.  Included by
// lbm_batch.cu only.
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
#pragma once

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
    if constexpr (RND) w.set_step(step);
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
            if constexpr (RND) w.set_step(t0[t.grid] + (uint32_t)k);
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
