// Host-side internals of liblbm.so shared by its translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/lbm.h"
#include "lbm_device.cuh"

namespace vss {

// Status of a launch helper: cudaSuccess or the CUDA error.
using Err = cudaError_t;

struct TileCfg {
    int vec = 4;     // sites per lane
    int rows = 16;   // rows per warp strip
    int warps = 4;   // warps per block
    int stages = 0;  // 2..4: bulk-copy row pipeline with this many stages (used
                     // when vec is 16 bytes of elements); 1: register walk with
                     // one row of loads prefetched (used when vec is 8 bytes of
                     // elements); 0: register walk
    // The default configuration: the register walks may change the tile
    // height at launch to fit the grid's tiles to the resident warps
    // (lbm_set_config and the tuner fix it).
    bool fit_rows = true;
};

// Sites per lane of the bulk-copy pipeline (16 bytes of elements).
inline int tma_vec(int storage) { return storage == ST_F32 ? 4 : 8; }
inline bool uses_tma(int storage, const TileCfg &c) {
    return c.stages >= 2 && c.vec == tma_vec(storage);
}
// Sites per lane of the prefetching register walk (8 bytes of elements).
inline int prefetch_vec(int storage) { return storage == ST_F32 ? 2 : 4; }
inline bool uses_prefetch(int storage, const TileCfg &c) {
    return c.stages == 1 && (c.vec == prefetch_vec(storage) || (storage != ST_F32 && c.vec == 8));
}

struct StepGeom {
    int nstrips, nsegs;
    long long ntiles;
};

inline StepGeom step_geom(int nx, int ny, const TileCfg &c) {
    StepGeom g;
    int w = 32 * c.vec;
    g.nstrips = (nx + w - 1) / w;
    g.nsegs = (ny + c.rows - 1) / c.rows;
    g.ntiles = (long long)g.nstrips * g.nsegs;
    return g;
}

// Element size in bytes of a storage kind.
inline int elem_bytes(int storage) { return storage == ST_F32 ? 4 : 2; }

// Plane stride in elements: nx*ny rounded up to 64 elements.
inline size_t plane_elems(int nx, int ny) {
    size_t n = (size_t)nx * (size_t)ny;
    return (n + 63) / 64 * 64;
}

Coef make_coef(double tau, double c2, double rho0);

// Kernel launchers (lbm_kernels.cu).  All asynchronous on `st`.
// `status` (device int) receives STATUS_TIMEOUT if a pipeline wait runs out.
// rnd = 1: stochastic rounding of 16-bit stores, seeded by the step number
// (*tdev if tdev is not NULL, plus toff).
// a15f: NULL for a uniform alpha, else 1.5 alpha per site ([ny][nx] floats).
Err launch_step(int storage, const TileCfg &cfg, const void *fin, void *fout, int nx, int ny,
                size_t P, const Coef &c, int *status, int rnd, const uint32_t *tdev, uint32_t toff,
                const float *a15f, cudaStream_t st);
// The forward-difference gradient (lbm_set_gradient): FP32, one site per lane.
Err launch_step_forward(const TileCfg &cfg, const void *fin, void *fout, int nx, int ny, size_t P,
                        const Coef &c, cudaStream_t st);
Err launch_a15_from_c2(const double *c2, float *a15, long long n, cudaStream_t st);
Err launch_set_u32(uint32_t *p, uint32_t v, cudaStream_t st);
// Sets the kernel attributes a configuration needs (dynamic shared memory);
// call before the first launch or capture of that configuration.
Err prepare_step(int storage, const TileCfg &cfg);
Err launch_init(int storage, void *f, int nx, int ny, size_t P, double rho0, const double *rho,
                const double *ux, const double *uy, cudaStream_t st);
// Driven-channel boundary columns (Section 4, Fig. 1 runs) on the buffer a
// step just wrote; step number *tdev + toff (tdev may be NULL).
Err launch_drive_x(int storage, void *f, int nx, int ny, size_t P, double rho0, double amp,
                   double period, const uint32_t *tdev, uint32_t toff, cudaStream_t st);
Err launch_moments(int storage, const void *f, int nx, int ny, size_t P, double rho0, double *rho,
                   double *ux, double *uy, cudaStream_t st);
// FP64 reductions: `partials` holds reduce_blocks(nx, ny) entries of the
// output's width (at most kReduceBlocksMax); `out` (device) receives the
// result values.
constexpr int kReduceBlocksMax = 1024;
int reduce_blocks(int nx, int ny);
Err launch_sums(int storage, const void *f, int nx, int ny, size_t P, double *partials,
                double *out3, cudaStream_t st);
Err launch_mode(int storage, const void *f, int nx, int ny, size_t P, double rho0, int field,
                int kx, int ky, double *partials, double *out2, cudaStream_t st);

bool valid_vec(int storage, int nx, int vec);

void set_error(const std::string &msg);

}  // namespace vss

// A grid handle (the opaque lbm_t of lbm.h).
struct lbm_grid {
    int nx = 0, ny = 0, storage = 0;
    double tau = 0, c2 = 0, rho0 = 1;
    size_t P = 0;                 // plane stride (elements)
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;                  // buf[cur] holds the state
    long long t = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    vss::Coef coef{};
    vss::TileCfg cfg{};
    int rounding = 0;             // 1: stochastic rounding of 16-bit stores
    float *a15f = nullptr;        // spatially varying alpha: 1.5 alpha per site
    int grad = 0;                 // LBM_GRAD_CENTRAL or LBM_GRAD_FORWARD
    // Slab of a grid decomposed in y (lbm_slab_create): this many ghost rows
    // at each end of the local buffer, which steps read but never compute
    // (0 for an ordinary periodic grid).
    int slab = 0;
    // Driven channel in x (lbm_set_drive): boundary columns after every step.
    bool drive = false;
    double drive_amp = 0, drive_period = 0;
    double *scratch = nullptr;    // reduction partials + results
    double *host_out = nullptr;   // pinned, 8 doubles
    // CUDA graphs of 2*graph_pairs steps starting from buffer 0 or buffer 1
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_pairs = 0;
    // Long step calls run as one persistent launch through a batch holding
    // only this grid (created on first use, dropped when the tiling changes).
    int persistent = LBM_PERSISTENT_AUTO;
    struct lbm_batch *self_batch = nullptr;
    // timing
    bool timing = false;
    double kernel_ms = 0;
    long long kernel_launches = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaEvent_t staged = nullptr;  // lbm_init: host fields copied
};

// Status word of a batch's kernels: batch_queue_status queues its copy to
// pinned host memory on `st`; once `st` has been synchronised, batch_status
// returns it (LBM_OK or LBM_ETIMEOUT).  Defined in lbm_batch.cu.
cudaError_t batch_queue_status(struct lbm_batch *b, cudaStream_t st);
int batch_status(const struct lbm_batch *b);
