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
    // Tiles of the grid in the work-list (flow schedule): the first one, how
    // many per step (segment-major: t = segment * nstrips + strip), and how
    // many segments / strips on each side a tile's step reads from (1, or 2
    // when a neighbouring segment or strip can be a single row or column).
    int tile0, ntile, nstrips, nsegs, dseg, dstrip;
};

// A tile: one strip (x0) of one segment (rows y0 .. y1-1, walked in
// direction dir) of a grid.  A paired tile (y1b > y0b; lockstep kernels of
// 8-site 16-bit walks only) adds a second segment, rows y0b .. y1b-1 in
// direction dirb, of a grid at most 16*8 columns wide: the two halves of the
// warp walk one segment each (the split walk).
struct __align__(16) Tile {
    int grid, x0, y0, y1, dir;
    int y0b, y1b, dirb;
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

// A 256-column tile of an 8-site 16-bit grid with a c2 field, in the general
// kernel: two 4-site walks of 128 columns (the register walk at 8 sites with
// the field's eight values spills heavily out of line; the results are the
// same bit for bit).
template <int S>
__device__ __forceinline__ void field_tile8(const GridDesc &g, int par, const Tile &t,
                                            uint32_t step) {
    do_tile<S, 4, true, 0, 1>(g, par, t, step);
    if (t.x0 + 128 < g.nx) {
        Tile u = t;
        u.x0 = t.x0 + 128;
        do_tile<S, 4, true, 0, 1>(g, par, u, step);
    }
}

// One tile of any kind (the walks out of line: one kernel for every mix).
__device__ __forceinline__ void any_tile(const GridDesc &g, int par, const Tile &t,
                                         uint32_t step) {
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
        case kind_code(ST_F16, 8, 0, 1):
            field_tile8<ST_F16>(g, par, t, step);
            break;
        case kind_code(ST_F16, 4, 0, 1):
            do_tile<ST_F16, 4, true, 0, 1>(g, par, t, step);
            break;
        case kind_code(ST_F16, 1, 0, 1):
            do_tile<ST_F16, 1, false, 0, 1>(g, par, t, step);
            break;
        case kind_code(ST_BF16, 8, 0, 1):
            field_tile8<ST_BF16>(g, par, t, step);
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
            any_tile(g, par, t, step);
        }
        if (k + 1 < nsteps && !grid_barrier(bar, status, timeout_ns)) return;
    }
}

// ---------------------------------------------------------------------------
// Flow schedule: every grid advances its own steps, with no barrier across
// the batch.  Each grid hands out tickets m = k * ntile + t (step k, tile t)
// from its own counter, in step order.  A warp holding (k, t) waits until
// every tile its step reads from or overwrites (the tiles within dseg
// segments and dstrip strips, wrapped, itself included) has completed step
// k - 1, runs the tile, and publishes k + 1 completed steps for it.  All
// tickets a wait depends on are earlier tickets of the same grid, already
// taken by warps that are running and never wait on later ones, so the
// kernel needs no co-residency guarantee and cannot deadlock.
//
// Warps pick grids round-robin, so every grid gets about the same number of
// tiles per unit time: small grids take many steps while large ones take
// few, instead of every grid waiting for the whole batch at every step.  A
// grid's tickets may run at most kFlowWindow steps ahead of its completed
// tiles, so that the warps a short grid's step chain would hold waiting go to
// other grids.
//
// Control words (zeroed before each launch): per grid, tickets taken and
// tiles completed (64-bit, each on its own 128-byte line); globally the
// round-robin counter and the number of grids whose last ticket is taken.
// Every wait is bounded by the same wall-clock limit as the barrier.
constexpr int kFlowWindow = 2;
constexpr int kFlowCtlWords = 32;  // unsigned long long words per grid: [0] taken, [16] done
constexpr int kFlowRR = 0;         // words of `glob`
constexpr int kFlowExh = 32;

__device__ __forceinline__ int wrap_idx(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

// Waits until the tiles step k of tile (seg, strip) depends on have
// completed k steps.  False if the wait ran out or another warp reported one.
__device__ __forceinline__ bool flow_wait(const GridDesc &g, const int *prog, int seg, int strip,
                                          int k, int *status, unsigned long long timeout_ns) {
    if (k == 0) return true;
    const int lane = threadIdx.x & 31;
    const int ns = 2 * g.dseg + 1, nt = 2 * g.dstrip + 1;
    int idx = -1;
    if (lane < ns * nt) {
        const int sq = wrap_idx(seg + lane / nt - g.dseg, g.nsegs);
        const int st = wrap_idx(strip + lane % nt - g.dstrip, g.nstrips);
        idx = g.tile0 + sq * g.nstrips + st;
    }
    unsigned long long t0 = 0;
    unsigned ns_sleep = 32;
    for (unsigned it = 0;; ++it) {
        const bool ok = idx < 0 || *(volatile const int *)(prog + idx) >= k;
        if (__all_sync(FULL, ok)) break;
        if (it == 0) t0 = global_ns();
        if ((it & 7u) == 7u) {
            int bad = 0;
            if (lane == 0) {
                if (*(volatile int *)status != 0) {
                    bad = 1;
                } else if (global_ns() - t0 > timeout_ns) {
                    atomicCAS(status, 0, LBM_ETIMEOUT);
                    bad = 1;
                }
            }
            if (__shfl_sync(FULL, bad, 0)) return false;
        }
        __nanosleep(ns_sleep);
        if (ns_sleep < 512u) ns_sleep *= 2u;
    }
    __threadfence();  // the flags are read before the tiles' data
    return true;
}

// The flow loop of one warp; run_tile(g, par, tile, step) runs a tile.
template <class RunTile>
__device__ __forceinline__ void flow_loop(const GridDesc *__restrict__ grids, int ngrids,
                                          const Tile *__restrict__ tiles,
                                          const long long *__restrict__ limit,
                                          const int *__restrict__ parity0,
                                          const uint32_t *__restrict__ t0,
                                          unsigned long long *ctl, int *prog, unsigned *glob,
                                          const int *__restrict__ nwork_p, int *status,
                                          unsigned long long timeout_ns, RunTile run_tile) {
    const int lane = threadIdx.x & 31;
    // The warp's ticket and idle timer live in shared memory while a tile
    // runs, leaving the walk the registers it has in the lockstep kernels.
    __shared__ unsigned long long idle_sh[kBatchWarps];
    __shared__ int tk_sh[kBatchWarps][3];
    const int wib = threadIdx.x >> 5;
    if (lane == 0) idle_sh[wib] = 0;
    __syncwarp();
    for (;;) {
        // Lane 0 takes a ticket from the next grid round-robin that has
        // tickets left and room in its window; -1: none right now; -2: done.
        int gsel = -1;
        unsigned long long m = 0;
        if (lane == 0) {
            if (*(volatile int *)status != 0) {
                gsel = -2;
            } else {
                const unsigned start = atomicAdd(glob + kFlowRR, 1u);
                for (int j = 0; j < ngrids && gsel == -1; ++j) {
                    const int cand = (int)((start + (unsigned)j) % (unsigned)ngrids);
                    const GridDesc &G = grids[cand];
                    const unsigned long long total =
                        (unsigned long long)limit[cand] * (unsigned long long)G.ntile;
                    volatile unsigned long long *c = ctl + (size_t)cand * kFlowCtlWords;
                    const unsigned long long taken = c[0];
                    if (taken >= total) continue;
                    if (taken - c[16] >= (unsigned long long)kFlowWindow * G.ntile) continue;
                    const unsigned long long mm =
                        atomicAdd(ctl + (size_t)cand * kFlowCtlWords, 1ULL);
                    if (mm >= total) continue;
                    if (mm + 1 == total) atomicAdd(glob + kFlowExh, 1u);
                    gsel = cand;
                    m = mm;
                }
                if (gsel == -1 && *(volatile unsigned *)(glob + kFlowExh) >= (unsigned)*nwork_p)
                    gsel = -2;
            }
        }
        gsel = __shfl_sync(FULL, gsel, 0);
        if (gsel == -2) return;
        if (gsel == -1) {
            // Every grid with tickets left is at the end of its window: wait
            // for tiles to complete (bounded, in case progress has stopped).
            int bad = 0;
            if (lane == 0) {
                const unsigned long long now = global_ns();
                if (idle_sh[wib] == 0) {
                    idle_sh[wib] = now;
                } else if (now - idle_sh[wib] > timeout_ns) {
                    atomicCAS(status, 0, LBM_ETIMEOUT);
                    bad = 1;
                }
            }
            if (__shfl_sync(FULL, bad, 0)) return;
            __nanosleep(256);
            continue;
        }
        m = __shfl_sync(FULL, m, 0);
        {
            const GridDesc &g = grids[gsel];
            const int k = (int)(m / (unsigned long long)g.ntile);
            const int ti = (int)(m % (unsigned long long)g.ntile);
            if (lane == 0) {
                idle_sh[wib] = 0;
                tk_sh[wib][0] = gsel;
                tk_sh[wib][1] = k;
                tk_sh[wib][2] = g.tile0 + ti;
            }
            const int seg = ti / g.nstrips, strip = ti % g.nstrips;
            if (!flow_wait(g, prog, seg, strip, k, status, timeout_ns)) return;
            const Tile t = tiles[g.tile0 + ti];
            run_tile(g, (parity0[gsel] + k) & 1, t, t0[gsel] + (uint32_t)k);
        }
        // Publish: the tile's stores before its completed-step count.
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            *(volatile int *)(prog + tk_sh[wib][2]) = tk_sh[wib][1] + 1;
            atomicAdd(ctl + (size_t)tk_sh[wib][0] * kFlowCtlWords + 16, 1ULL);
        }
    }
}

// Flow kernel for any mix of walks (out of line, as in k_batch).
__global__ void __launch_bounds__(32 * kBatchWarps, 3)
    k_flow(const GridDesc *__restrict__ grids, int ngrids, const Tile *__restrict__ tiles,
           const long long *__restrict__ limit, const int *__restrict__ parity0,
           const uint32_t *__restrict__ t0, unsigned long long *ctl, int *prog, unsigned *glob,
           const int *__restrict__ nwork_p, int *status, unsigned long long timeout_ns) {
    flow_loop(grids, ngrids, tiles, limit, parity0, t0, ctl, prog, glob, nwork_p, status,
              timeout_ns, [](const GridDesc &g, int par, const Tile &t, uint32_t step) {
                  any_tile(g, par, t, step);
              });
}

// Flow kernel for a batch of one walk, inlined (the register budget and the
// row buffers of k_batch_one: 16 warps per SM, measured faster than 12
// without spills although the flow loop's state costs a few bytes of spill).
template <int S, int V, int PD, int RND, int VA = 0>
__global__ void __launch_bounds__(32 * kBatchWarps, PD == 2 ? 3 : 4)
    k_flow_one(const GridDesc *__restrict__ grids, int ngrids, const Tile *__restrict__ tiles,
               const long long *__restrict__ limit, const int *__restrict__ parity0,
               const uint32_t *__restrict__ t0, unsigned long long *ctl, int *prog,
               unsigned *glob, const int *__restrict__ nwork_p, int *status,
               unsigned long long timeout_ns) {
    __shared__ uint4 rowbuf[(S != ST_F32 && V == 8) ? kBatchWarps : 1][(2 * 9 + (VA ? 4 : 0)) * 32];
    (void)rowbuf;
    flow_loop(grids, ngrids, tiles, limit, parity0, t0, ctl, prog, glob, nwork_p, status,
              timeout_ns, [&](const GridDesc &g, int par, const Tile &t, uint32_t step) {
                  Walker<S, V, LD_CG, RND, VA> w(g.buf[par], g.buf[par ^ 1], g.nx, g.ny, g.P,
                                                 t.x0);
                  if constexpr (VA) w.a15f = g.a15f;
                  if constexpr (RND) w.set_step(step);
                  const Coef c = g.c;
                  if constexpr (S != ST_F32 && V == 8)
                      w.run_async(t.y0, t.y1, t.dir, c, &rowbuf[threadIdx.x >> 5][0]);
                  else if constexpr (PD == 2)
                      w.run_prefetch2(t.y0, t.y1, t.dir, c);
                  else if constexpr (PD == 1)
                      w.run_prefetch(t.y0, t.y1, t.dir, c);
                  else
                      w.run(t.y0, t.y1, t.dir, c);
              });
}

// Flow kernel for the serving mix: FP32 grids (4 sites per lane) and 16-bit
// grids of storage S2 and rounding RND2 (8 sites per lane), both walks
// inlined; 12 warps per SM (at 16 both walks together spill heavily).
template <int S2, int RND2>
__global__ void __launch_bounds__(32 * kBatchWarps, 3)
    k_flow_two(const GridDesc *__restrict__ grids, int ngrids, const Tile *__restrict__ tiles,
               const long long *__restrict__ limit, const int *__restrict__ parity0,
               const uint32_t *__restrict__ t0, unsigned long long *ctl, int *prog,
               unsigned *glob, const int *__restrict__ nwork_p, int *status,
               unsigned long long timeout_ns) {
    __shared__ uint4 rowbuf[kBatchWarps][2 * 9 * 32];
    flow_loop(grids, ngrids, tiles, limit, parity0, t0, ctl, prog, glob, nwork_p, status,
              timeout_ns, [&](const GridDesc &g, int par, const Tile &t, uint32_t step) {
                  const Coef c = g.c;
                  if (g.kind == kind_code(ST_F32, 4, 0)) {
                      Walker<ST_F32, 4, LD_CG> w(g.buf[par], g.buf[par ^ 1], g.nx, g.ny, g.P,
                                                 t.x0);
                      w.run(t.y0, t.y1, t.dir, c);
                  } else {
                      Walker<S2, 8, LD_CG, RND2> w(g.buf[par], g.buf[par ^ 1], g.nx, g.ny, g.P,
                                                   t.x0);
                      if constexpr (RND2) w.set_step(step);
                      w.run_async(t.y0, t.y1, t.dir, c, &rowbuf[threadIdx.x >> 5][0]);
                  }
              });
}

using FlowKernel = void (*)(const GridDesc *, int, const Tile *, const long long *, const int *,
                            const uint32_t *, unsigned long long *, int *, unsigned *,
                            const int *, int *, unsigned long long);

// The flow kernel for a batch's kinds: specialised when all grids share one
// walk, else the general k_flow.
FlowKernel flow_kernel_for(const std::vector<int> &kinds, int walk16) {
    bool same = true;
    for (int k : kinds) same = same && k == kinds[0];
    if (!kinds.empty() && same) {
        const bool two = walk16 == LBM_WALK16_V4_PF2;
        switch (kinds[0]) {
            case kind_code(ST_F32, 4, 0):
                return k_flow_one<ST_F32, 4, 0, 0>;
            case kind_code(ST_F16, 8, 0):
                return k_flow_one<ST_F16, 8, 0, 0>;
            case kind_code(ST_BF16, 8, 0):
                return k_flow_one<ST_BF16, 8, 0, 0>;
            case kind_code(ST_F16, 8, 1):
                return k_flow_one<ST_F16, 8, 0, 1>;
            case kind_code(ST_BF16, 8, 1):
                return k_flow_one<ST_BF16, 8, 0, 1>;
            case kind_code(ST_F16, 4, 0):
                return two ? k_flow_one<ST_F16, 4, 2, 0> : k_flow_one<ST_F16, 4, 1, 0>;
            case kind_code(ST_BF16, 4, 0):
                return two ? k_flow_one<ST_BF16, 4, 2, 0> : k_flow_one<ST_BF16, 4, 1, 0>;
            case kind_code(ST_F32, 4, 0, 1):
                return k_flow_one<ST_F32, 4, 0, 0, 1>;
            default:
                break;
        }
    }
    // FP32 (4 sites per lane) with one 16-bit kind of 8 sites per lane.
    int other = -1;
    bool pair = !kinds.empty();
    for (int k : kinds) {
        if (k == kind_code(ST_F32, 4, 0)) continue;
        if (other == -1) other = k;
        pair = pair && k == other;
    }
    if (pair && other != -1) {
        switch (other) {
            case kind_code(ST_F16, 8, 0):
                return k_flow_two<ST_F16, 0>;
            case kind_code(ST_BF16, 8, 0):
                return k_flow_two<ST_BF16, 0>;
            case kind_code(ST_F16, 8, 1):
                return k_flow_two<ST_F16, 1>;
            case kind_code(ST_BF16, 8, 1):
                return k_flow_two<ST_BF16, 1>;
            default:
                break;
        }
    }
    return k_flow;
}

// Walks whose lockstep kernel takes paired tiles (the split walk): 8-site
// 16-bit walks without a c2 field.  kind_splits is the same test on a kind
// code, for the work-list builder.
template <int S, int V, int VA>
constexpr bool kSplitWalk = S != ST_F32 && V == 8 && VA == 0;
constexpr bool kind_splits(int kd) {
    return kd == kind_code(ST_F16, 8, 0) || kd == kind_code(ST_BF16, 8, 0) ||
           kd == kind_code(ST_F16, 8, 1) || kd == kind_code(ST_BF16, 8, 1);
}
constexpr int kSplitCols = 16 * 8;     // widest grid a half-warp walks
constexpr double kSplitMinShare = 0.2;  // of a group's tiles, for the split kernel

// A paired tile: each half-warp walks its own segment of the grid.  Inlined:
// out of line, the call made both walks slower (measured).
template <int S, int RND>
__device__ __forceinline__ void split_tile(const GridDesc &g, int par, const Tile &t,
                                           uint32_t step, uint4 *buf) {
    Walker<S, 8, LD_CG, RND, 0, 16> w(g.buf[par], g.buf[par ^ 1], g.nx, g.ny, g.P, t.x0);
    if constexpr (RND) w.set_step(step);
    const bool hi = (threadIdx.x & 16) != 0;
    const int K = max(t.y1 - t.y0, t.y1b - t.y0b) + 2;
    const Coef c = g.c;
    w.run_async_split(hi ? t.y0b : t.y0, hi ? t.y1b : t.y1, hi ? t.dirb : t.dir, K, c, buf);
}

// Specialised persistent kernel for a batch whose grids all use one walk
// (storage, vec, rounding, rows of loads in flight PD = 0, 1 or 2): the walk is
// inlined, so the kernel keeps the single-grid kernel's register budget (128,
// 16 warps per SM; 170 and 12 warps per SM for the two-row prefetch) instead
// of paying for calls.  Same time-step loop and bounded barrier as k_batch.
template <int S, int V, int PD, int RND, int VA = 0, bool SPLIT = false>
__global__ void __launch_bounds__(32 * kBatchWarps, PD == 2 ? 3 : 4)
    k_batch_one(const GridDesc *__restrict__ grids, const Tile *__restrict__ tiles, int ntiles,
                const long long *__restrict__ limit, const int *__restrict__ parity0,
                const uint32_t *__restrict__ t0, long long nsteps, unsigned *bar, int *status,
                unsigned long long timeout_ns) {
    // Row buffers of the 8-site 16-bit walks: per warp a landing slot and a
    // stash of 9 x 32 16-byte vectors each (36 KiB per block), and with a c2
    // field two slots of 2 x 32 vectors for its values (44 KiB per block).
    __shared__ uint4 rowbuf[(S != ST_F32 && V == 8) ? kBatchWarps : 1][(2 * 9 + (VA ? 4 : 0)) * 32];
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
            if constexpr (SPLIT) {
                static_assert(kSplitWalk<S, V, VA>, "paired tiles need the 8-site 16-bit walk");
                if (t.y1b > t.y0b) {
                    split_tile<S, RND>(g, par, t, t0[t.grid] + (uint32_t)k,
                                       &rowbuf[threadIdx.x >> 5][0]);
                    continue;
                }
            }
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
// `split`: the tiles include paired ones (8-site 16-bit kinds only), run by
// the kernel instance that has the split walk.
BatchKernel kernel_for(const std::vector<int> &kinds, int walk16, bool split = false) {
    bool same = true;
    for (int k : kinds) same = same && k == kinds[0];
    if (!kinds.empty() && same) {
        const bool two = walk16 == LBM_WALK16_V4_PF2;
        switch (kinds[0]) {
            case kind_code(ST_F32, 4, 0):
                return k_batch_one<ST_F32, 4, 0, 0>;
            case kind_code(ST_F16, 8, 0):
                return split ? k_batch_one<ST_F16, 8, 0, 0, 0, true> : k_batch_one<ST_F16, 8, 0, 0>;
            case kind_code(ST_BF16, 8, 0):
                return split ? k_batch_one<ST_BF16, 8, 0, 0, 0, true>
                             : k_batch_one<ST_BF16, 8, 0, 0>;
            case kind_code(ST_F16, 8, 1):
                return split ? k_batch_one<ST_F16, 8, 0, 1, 0, true> : k_batch_one<ST_F16, 8, 0, 1>;
            case kind_code(ST_BF16, 8, 1):
                return split ? k_batch_one<ST_BF16, 8, 0, 1, 0, true>
                             : k_batch_one<ST_BF16, 8, 0, 1>;
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
            case kind_code(ST_F16, 8, 0, 1):
                return k_batch_one<ST_F16, 8, 0, 0, 1>;
            case kind_code(ST_BF16, 8, 0, 1):
                return k_batch_one<ST_BF16, 8, 0, 0, 1>;
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
