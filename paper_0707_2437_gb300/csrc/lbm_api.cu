// C ABI of liblbm.so: handles, validation, streams, ping-pong buffers, CUDA
// graphs of step sequences, checkpoints, the tile autotuner and error codes.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace vss;

// ---------------------------------------------------------------------------
// Errors.

static thread_local std::string g_last_error;

namespace vss {
void set_error(const std::string &msg) { g_last_error = msg; }
}  // namespace vss

static int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

static int cuda_fail(cudaError_t e, const char *where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

extern "C" const char *lbm_strerror(int status) {
    switch (status) {
        case LBM_OK:
            return "ok";
        case LBM_EINVAL:
            return "invalid argument";
        case LBM_ENOMEM:
            return "out of memory";
        case LBM_ECUDA:
            return "CUDA error";
        case LBM_ENONFINITE:
            return "non-finite value in a reduction";
        case LBM_ETIMEOUT:
            return "in-kernel wait timed out";
        case LBM_WUNSTABLE:
            return "warning: sound speed above the largest stable value observed (c_e > 1.125)";
        default:
            return "unknown status";
    }
}

extern "C" const char *lbm_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// Handle.

static size_t state_bytes(const lbm_grid *h) { return 9 * h->P * (size_t)elem_bytes(h->storage); }

// Defaults from measured steps: FP32 runs fastest as the plain register walk
// with 128-bit vectors; the 16-bit kinds as the 8-site walk with rows through
// shared memory when nx is a multiple of 8 and its 16-row tiles fill at least
// a quarter of the resident warps (16 per SM), else as the prefetching
// register walk with 64-bit vectors (per step, 256-step calls: 2048^2 FP16-delta
// 25.4 us against 29.8, 8192^2 372.7 against 405.7; 1024^2 10.1 against 8.8,
// its 8-site tiles fitting only at 2 rows).  Narrower vectors serve grids whose
// nx they do not divide.
static TileCfg default_cfg(int storage, int nx, int ny, int sms) {
    TileCfg c;
    c.rows = 16;
    c.warps = 4;
    c.stages = 0;
    if (storage == ST_F32) {
        c.vec = 1;
        for (int v = 4; v >= 1; v /= 2)
            if (valid_vec(storage, nx, v)) {
                c.vec = v;
                break;
            }
    } else if (valid_vec(storage, nx, 8) &&
               4LL * ((nx + 255) / 256) * ((ny + 15) / 16) >= 16LL * sms) {
        c.vec = 8;  // k_step_async
    } else if (valid_vec(storage, nx, prefetch_vec(storage))) {
        c.vec = prefetch_vec(storage);
        c.stages = 1;
    } else {
        c.vec = nx % 2 == 0 ? 2 : 1;
    }
    return c;
}

// Device status word written by kernels whose bounded waits ran out.
static int *status_ptr(lbm_grid *h) { return reinterpret_cast<int *>(h->scratch + 8); }
// Device step counter that seeds stochastic rounding inside graph replays.
static uint32_t *step_ptr(lbm_grid *h) { return reinterpret_cast<uint32_t *>(h->scratch + 9); }

// Waits for the grid's stream once and returns the status of the work on it:
// the copies of the step kernels' status word and of the grid's own
// persistent batch's status word to pinned host memory are queued first, so
// one synchronisation serves the caller's results and the status.  A set
// status word is cleared (stream-ordered) and returned as the error.
static int sync_status(lbm_grid *h) {
    int *hs = reinterpret_cast<int *>(h->host_out + 7);
    CK(cudaMemcpyAsync(hs, status_ptr(h), sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    if (h->self_batch) CK(batch_queue_status(h->self_batch, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (h->self_batch) {
        int rb = batch_status(h->self_batch);
        if (rb != LBM_OK) return fail(rb, "a barrier wait in the persistent step kernel ran out");
    }
    if (*hs != 0) {
        int st = *hs;
        cudaMemsetAsync(status_ptr(h), 0, sizeof(int), h->stream);
        return fail(st, "a bounded wait in the step kernel ran out");
    }
    return LBM_OK;
}

static void drop_self_batch(lbm_grid *h) {
    if (h->self_batch) {
        lbm_batch_destroy(h->self_batch);
        h->self_batch = nullptr;
    }
}

static void drop_graphs(lbm_grid *h) {
    for (int k = 0; k < 2; ++k)
        if (h->graph[k]) {
            cudaGraphExecDestroy(h->graph[k]);
            h->graph[k] = nullptr;
        }
    h->graph_pairs = 0;
}

// ---------------------------------------------------------------------------
// Staging memory for host fields (lbm_init) and host moments (lbm_moments).
// It comes from a pool owned by the library, one per device, that keeps up
// to kStagingKeep bytes reserved across synchronisations.  The default pool
// returns freed memory to the system at every synchronisation, and mapping it
// again on the next call costs more than the copies it serves.  When a grid's
// buffers do not fit, the pool is trimmed and the allocation retried.

static constexpr unsigned long long kStagingKeep = 1ull << 30;
static std::mutex g_pool_mu;
static std::map<int, cudaMemPool_t> g_pools;

// Per-device stream for lbm_init's host-to-device copies.  The copies do not
// queue behind the work on the grid's stream (a running batch, say), so the
// call returns as soon as the host fields are read; the grid's stream waits
// for the copies before the initialisation kernel.
static std::map<int, cudaStream_t> g_copy_streams;

static cudaError_t copy_stream(int device, cudaStream_t *out) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_copy_streams.find(device);
    if (it != g_copy_streams.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    // Created on the grid's device, whichever device is current.
    int cur = device;
    cudaError_t e = cudaGetDevice(&cur);
    if (e == cudaSuccess && cur != device) e = cudaSetDevice(device);
    cudaStream_t s = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess) return e;
    g_copy_streams[device] = s;
    *out = s;
    return cudaSuccess;
}

static cudaError_t staging_alloc(lbm_grid *h, double **p, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        auto it = g_pools.find(h->device);
        if (it != g_pools.end()) {
            pool = it->second;
        } else {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = h->device;
            cudaError_t e = cudaMemPoolCreate(&pool, &props);
            if (e != cudaSuccess) return e;
            unsigned long long keep = kStagingKeep;
            e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            // Memory freed on one stream is reused on another only once the
            // free has completed: the pool never makes the copy stream wait
            // for a grid's stream.
            int no = 0;
            if (e == cudaSuccess)
                e = cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
            if (e != cudaSuccess) {
                cudaMemPoolDestroy(pool);
                return e;
            }
            g_pools[h->device] = pool;
        }
    }
    return cudaMallocFromPoolAsync(reinterpret_cast<void **>(p), bytes, pool, st);
}

// Returns the staging pool's unused reservation of `device` to the system.
static void trim_staging(int device) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(device);
    if (it != g_pools.end()) {
        cudaDeviceSynchronize();
        cudaMemPoolTrimTo(it->second, 0);
    }
}

extern "C" size_t lbm_bytes_required(int nx, int ny, int storage) {
    if (nx < 1 || ny < 1 || storage < 0 || storage > 2) return 0;
    if ((long long)nx * ny > 0x7fffffffLL) return 0;
    return 2 * 9 * plane_elems(nx, ny) * (size_t)elem_bytes(storage);
}

extern "C" int lbm_mem_info(size_t *free_bytes, size_t *total_bytes) {
    size_t f = 0, t = 0;
    CK(cudaMemGetInfo(&f, &t));
    if (free_bytes) *free_bytes = f;
    if (total_bytes) *total_bytes = t;
    return LBM_OK;
}

extern "C" int lbm_create_ex(int nx, int ny, double tau, double c2, double rho0, int storage,
                             void *cuda_stream, lbm_t *out) {
    if (!out) return fail(LBM_EINVAL, "lbm_create: out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || (long long)nx * ny > 0x7fffffffLL)
        return fail(LBM_EINVAL, "lbm_create: need nx, ny >= 1 and nx*ny < 2^31");
    if (!(tau > 0.5) || !isfinite(tau)) return fail(LBM_EINVAL, "lbm_create: need tau > 0.5");
    if (!(c2 > 0.0) || !isfinite(c2)) return fail(LBM_EINVAL, "lbm_create: need c2 > 0");
    if (!(rho0 > 0.0) || !isfinite(rho0)) return fail(LBM_EINVAL, "lbm_create: need rho0 > 0");
    if (storage < 0 || storage > 2) return fail(LBM_EINVAL, "lbm_create: unknown storage");

    lbm_grid *h = new (std::nothrow) lbm_grid();
    if (!h) return fail(LBM_ENOMEM, "lbm_create: host allocation failed");
    h->nx = nx;
    h->ny = ny;
    h->tau = tau;
    h->c2 = c2;
    h->rho0 = rho0;
    h->storage = storage;
    h->P = plane_elems(nx, ny);
    h->stream = (cudaStream_t)cuda_stream;
    h->coef = make_coef(tau, c2, rho0);
    cudaError_t e = cudaGetDevice(&h->device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    h->cfg = default_cfg(storage, nx, ny, sms > 0 ? sms : 1);
    size_t bytes = state_bytes(h);
    if (e == cudaSuccess) e = cudaMalloc(&h->buf[0], bytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->buf[1], bytes);
    if (e == cudaErrorMemoryAllocation) {
        // Cached staging memory may be in the way: release it and retry.
        cudaGetLastError();
        trim_staging(h->device);
        e = cudaSuccess;
        if (!h->buf[0]) e = cudaMalloc(&h->buf[0], bytes);
        if (e == cudaSuccess && !h->buf[1]) e = cudaMalloc(&h->buf[1], bytes);
    }
    if (e == cudaSuccess) e = cudaMalloc(&h->scratch, sizeof(double) * (3 * 1024 + 16));
    // Stream-ordered, so that creating a grid does not wait for work running
    // on the legacy default stream.
    if (e == cudaSuccess) e = cudaMemsetAsync(h->scratch, 0, sizeof(double) * 16, h->stream);
    if (e == cudaSuccess) e = prepare_step(storage, h->cfg);
    if (e == cudaSuccess) e = cudaMallocHost(&h->host_out, sizeof(double) * 8);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev[1]);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->staged, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "lbm_create");
        lbm_destroy(h);
        cudaGetLastError();
        return rc;
    }
    *out = h;
    return c2 > 1.2656 ? LBM_WUNSTABLE : LBM_OK;
}

extern "C" int lbm_create(int nx, int ny, double tau, double c2, int storage, void *cuda_stream,
                          lbm_t *out) {
    return lbm_create_ex(nx, ny, tau, c2, 1.0, storage, cuda_stream, out);
}

extern "C" int lbm_destroy(lbm_t h) {
    if (!h) return LBM_OK;
    if (h->stream || h->buf[0]) cudaStreamSynchronize(h->stream);
    drop_self_batch(h);
    drop_graphs(h);
    for (int k = 0; k < 2; ++k) {
        if (h->buf[k]) cudaFree(h->buf[k]);
        if (h->ev[k]) cudaEventDestroy(h->ev[k]);
    }
    if (h->staged) cudaEventDestroy(h->staged);
    if (h->scratch) cudaFree(h->scratch);
    if (h->a15f) cudaFree(h->a15f);
    if (h->host_out) cudaFreeHost(h->host_out);
    delete h;
    return LBM_OK;
}

// Copies a [ny][nx] double field to device scratch on stream `cs` if it is
// on the host.
static int stage_field(lbm_grid *h, const double *src, int on_device, cudaStream_t cs,
                       double **dev, std::vector<double *> &owned) {
    if (on_device) {
        *dev = const_cast<double *>(src);
        return LBM_OK;
    }
    size_t n = (size_t)h->nx * h->ny;
    double *d = nullptr;
    CK(staging_alloc(h, &d, n * sizeof(double), cs));
    owned.push_back(d);
    CK(cudaMemcpyAsync(d, src, n * sizeof(double), cudaMemcpyHostToDevice, cs));
    *dev = d;
    return LBM_OK;
}

extern "C" int lbm_init(lbm_t h, const double *rho, const double *ux, const double *uy,
                        int on_device) {
    if (!h || !rho || !ux || !uy) return fail(LBM_EINVAL, "lbm_init: NULL argument");
    std::vector<double *> owned;
    double *dr = nullptr, *du = nullptr, *dv = nullptr;
    cudaStream_t cs = h->stream;
    if (!on_device) CK(copy_stream(h->device, &cs));
    int rc = stage_field(h, rho, on_device, cs, &dr, owned);
    if (rc == LBM_OK) rc = stage_field(h, ux, on_device, cs, &du, owned);
    if (rc == LBM_OK) rc = stage_field(h, uy, on_device, cs, &dv, owned);
    if (!on_device && !owned.empty()) {
        // The grid's stream waits for the copies (also when one failed, so
        // that the frees below stay ordered after them).
        cudaError_t e = cudaEventRecord(h->staged, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->staged, 0);
        if (e != cudaSuccess && rc == LBM_OK) rc = cuda_fail(e, "lbm_init");
    }
    if (rc == LBM_OK) {
        cudaError_t e = launch_init(h->storage, h->buf[0], h->nx, h->ny, h->P, h->rho0, dr, du, dv,
                                    h->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "lbm_init kernel");
    }
    for (double *p : owned) cudaFreeAsync(p, h->stream);
    if (rc != LBM_OK) return rc;
    h->cur = 0;
    h->t = 0;
    // Host fields: wait only until the copies have read them (they run on
    // the copy stream; the kernel stays queued on the grid's stream, so the
    // call does not wait for work ahead of it there).  Device fields: wait
    // until the kernel has read them.
    if (on_device)
        CK(cudaStreamSynchronize(h->stream));
    else
        CK(cudaEventSynchronize(h->staged));
    return LBM_OK;
}

// The driven-channel boundary columns for the step numbered *tdev + toff,
// written into the buffer that step produced.
static cudaError_t launch_drive(lbm_grid *h, void *out, const uint32_t *tdev, uint32_t toff,
                                cudaStream_t st) {
    return launch_drive_x(h->storage, out, h->nx, h->ny, h->P, h->rho0, h->drive_amp,
                          h->drive_period, tdev, toff, st);
}

// One step launch from buf[cur] to buf[cur ^ 1] (no bookkeeping), followed
// by the boundary columns when the channel is driven.
static cudaError_t launch_one(lbm_grid *h, int from) {
    cudaError_t e =
        h->grad == LBM_GRAD_FORWARD
            ? launch_step_forward(h->cfg, h->buf[from], h->buf[from ^ 1], h->nx, h->ny, h->P,
                                  h->coef, h->stream)
            : launch_step(h->storage, h->cfg, h->buf[from], h->buf[from ^ 1], h->nx, h->ny, h->P,
                          h->coef, status_ptr(h), h->rounding, nullptr, (uint32_t)h->t, h->a15f,
                          h->stream);
    if (e == cudaSuccess && h->drive)
        e = launch_drive(h, h->buf[from ^ 1], nullptr, (uint32_t)h->t, h->stream);
    return e;
}

static const int kGraphPairs = 16;   // a graph holds 32 steps
static const long long kPersistentMin = 64;  // persistent launch from this many steps
// ... or from kPersistentMinLarge steps on grids of at least kLargeSites sites,
// where a step is long enough that the launch's barrier costs little.
static const long long kPersistentMinLarge = 8;
static const long long kLargeSites = 1LL << 20;
static const long long kGraphMin = 8; // use graphs from this many steps on
// LBM_PERSISTENT_AUTO steps every grid with the step kernel (except slabs):
// per step over 256- and 1024-step calls it was the faster for FP32 grids from
// 64^2 to 8192^2 (2048^2 49.6 us against 52.2 persistent, 64^2 3.5 against
// 6.1), for 16-bit grids with its 8-site walk (2048^2 FP16-delta 25.4 against
// 30.8, 8192^2 372.7 against 384.8) and with a c2 field (4096^2 FP16-delta
// 125.7 against 131.2).

static int build_graphs(lbm_grid *h) {
    drop_graphs(h);
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    for (int start = 0; start < 2; ++start) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int k = 0; k < 2 * kGraphPairs && e == cudaSuccess; ++k) {
                e = h->grad == LBM_GRAD_FORWARD
                        ? launch_step_forward(h->cfg, h->buf[(start + k) & 1],
                                              h->buf[(start + k + 1) & 1], h->nx, h->ny, h->P,
                                              h->coef, cs)
                        : launch_step(h->storage, h->cfg, h->buf[(start + k) & 1],
                                      h->buf[(start + k + 1) & 1], h->nx, h->ny, h->P, h->coef,
                                      status_ptr(h), h->rounding, step_ptr(h), (uint32_t)k,
                                      h->a15f, cs);
                if (e == cudaSuccess && h->drive)
                    e = launch_drive(h, h->buf[(start + k + 1) & 1], step_ptr(h), (uint32_t)k, cs);
            }
            cudaError_t e2 = cudaStreamEndCapture(cs, &g);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph[start], g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cs);
            drop_graphs(h);
            return cuda_fail(e, "lbm_step: graph capture");
        }
    }
    cudaStreamDestroy(cs);
    h->graph_pairs = kGraphPairs;
    return LBM_OK;
}

extern "C" int lbm_step(lbm_t h, long long n) {
    if (!h || n < 0) return fail(LBM_EINVAL, "lbm_step: bad handle or n < 0");
    if (n == 0) return LBM_OK;
    if (h->timing) {
        // Per-launch events: accumulate device time of every launch.
        double total = 0.0;
        for (long long k = 0; k < n; ++k) {
            CK(cudaEventRecord(h->ev[0], h->stream));
            cudaError_t e = launch_one(h, h->cur);
            if (e != cudaSuccess) return cuda_fail(e, "lbm_step kernel");
            CK(cudaEventRecord(h->ev[1], h->stream));
            CK(cudaEventSynchronize(h->ev[1]));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
            total += ms;
            h->cur ^= 1;
            h->t += 1;
        }
        h->kernel_ms = total / (double)n;
        h->kernel_launches = n;
        return LBM_OK;
    }
    if (h->slab && n != 1)
        return fail(LBM_EINVAL, "lbm_step: a slab takes one step at a time (its ghost rows "
                                "are refreshed between steps)");
    const long long sites = (long long)h->nx * h->ny;
    bool persistent = false;
    if (h->persistent == LBM_PERSISTENT_ON)
        persistent = n >= kPersistentMin || (sites >= kLargeSites && n >= kPersistentMinLarge);
    if (h->slab || (persistent && !h->drive && h->grad == LBM_GRAD_CENTRAL)) {
        // Slabs always step here: the batch's tile list covers only their
        // own rows.
        // One persistent launch of all n steps (dynamic tile scheduling,
        // barrier between steps), bitwise the same as n single launches.
        if (!h->self_batch) {
            lbm_t self = h;
            int rc = lbm_batch_create(&self, 1, &h->self_batch);
            if (rc != LBM_OK) return rc;
        }
        return lbm_batch_step(h->self_batch, n, nullptr);  // advances t and cur
    }
    if (n >= kGraphMin) {
        if (!h->graph_pairs) {
            int rc = build_graphs(h);
            if (rc != LBM_OK) return rc;
        }
        long long per = 2LL * h->graph_pairs;
        while (n >= per) {
            if (h->rounding || h->drive)
                CK(launch_set_u32(step_ptr(h), (uint32_t)h->t, h->stream));
            CK(cudaGraphLaunch(h->graph[h->cur], h->stream));
            n -= per;
            h->t += per;  // an even number of steps leaves cur unchanged
        }
    }
    for (long long k = 0; k < n; ++k) {
        cudaError_t e = launch_one(h, h->cur);
        if (e != cudaSuccess) return cuda_fail(e, "lbm_step kernel");
        h->cur ^= 1;
        h->t += 1;
    }
    return LBM_OK;
}

extern "C" int lbm_set_persistent(lbm_t h, int on) {
    if (!h) return fail(LBM_EINVAL, "lbm_set_persistent: NULL handle");
    if (on != LBM_PERSISTENT_OFF && on != LBM_PERSISTENT_ON && on != LBM_PERSISTENT_AUTO)
        return fail(LBM_EINVAL, "lbm_set_persistent: unknown mode");
    CK(cudaStreamSynchronize(h->stream));
    h->persistent = on;
    if (on == LBM_PERSISTENT_OFF) drop_self_batch(h);
    return LBM_OK;
}

extern "C" int lbm_set_timing(lbm_t h, int on) {
    if (!h) return fail(LBM_EINVAL, "lbm_set_timing: NULL handle");
    h->timing = on != 0;
    return LBM_OK;
}

extern "C" int lbm_kernel_ms(lbm_t h, double *ms, long long *launches) {
    if (!h) return fail(LBM_EINVAL, "lbm_kernel_ms: NULL handle");
    if (ms) *ms = h->kernel_ms;
    if (launches) *launches = h->kernel_launches;
    return LBM_OK;
}

extern "C" int lbm_moments(lbm_t h, double *rho, double *ux, double *uy, int on_device) {
    if (!h) return fail(LBM_EINVAL, "lbm_moments: NULL handle");
    size_t n = (size_t)h->nx * h->ny;
    if (on_device) {
        cudaError_t e = launch_moments(h->storage, h->buf[h->cur], h->nx, h->ny, h->P, h->rho0,
                                       rho, ux, uy, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "lbm_moments kernel");
        return sync_status(h);
    }
    double *d = nullptr;
    CK(staging_alloc(h, &d, 3 * n * sizeof(double), h->stream));
    cudaError_t e = launch_moments(h->storage, h->buf[h->cur], h->nx, h->ny, h->P, h->rho0,
                                   rho ? d : nullptr, ux ? d + n : nullptr,
                                   uy ? d + 2 * n : nullptr, h->stream);
    if (e == cudaSuccess && rho)
        e = cudaMemcpyAsync(rho, d, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && ux)
        e = cudaMemcpyAsync(ux, d + n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && uy)
        e = cudaMemcpyAsync(uy, d + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost,
                            h->stream);
    cudaFreeAsync(d, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_moments");
    return sync_status(h);
}

extern "C" int lbm_sums(lbm_t h, double *out3) {
    if (!h || !out3) return fail(LBM_EINVAL, "lbm_sums: NULL argument");
    double *partials = h->scratch + 16;
    cudaError_t e = launch_sums(h->storage, h->buf[h->cur], h->nx, h->ny, h->P, partials,
                                h->scratch, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_sums kernel");
    CK(cudaMemcpyAsync(h->host_out, h->scratch, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream));
    int rs = sync_status(h);
    if (rs != LBM_OK) return rs;
    out3[0] = (double)h->nx * (double)h->ny * h->rho0 + h->host_out[0];
    out3[1] = h->host_out[1];
    out3[2] = h->host_out[2];
    for (int k = 0; k < 3; ++k)
        if (!isfinite(out3[k])) return fail(LBM_ENONFINITE, "lbm_sums: non-finite total");
    return LBM_OK;
}

extern "C" int lbm_mode(lbm_t h, int field, int kx, int ky, double *out2) {
    if (!h || !out2 || field < 0 || field > 2)
        return fail(LBM_EINVAL, "lbm_mode: bad argument");
    double *partials = h->scratch + 16;
    cudaError_t e = launch_mode(h->storage, h->buf[h->cur], h->nx, h->ny, h->P, h->rho0, field, kx,
                                ky, partials, h->scratch, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lbm_mode kernel");
    CK(cudaMemcpyAsync(h->host_out, h->scratch, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream));
    int rs = sync_status(h);
    if (rs != LBM_OK) return rs;
    out2[0] = h->host_out[0];
    out2[1] = h->host_out[1];
    if (!isfinite(out2[0]) || !isfinite(out2[1]))
        return fail(LBM_ENONFINITE, "lbm_mode: non-finite value");
    return LBM_OK;
}

extern "C" long long lbm_time(lbm_t h) { return h ? h->t : -1; }

extern "C" int lbm_set_stream(lbm_t h, void *cuda_stream) {
    if (!h) return fail(LBM_EINVAL, "lbm_set_stream: NULL handle");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (s == h->stream) return LBM_OK;
    if (h->self_batch) {
        // The grid's persistent batch runs on the old stream: its status is
        // taken and it is rebuilt on the new stream at the next long call.
        int rb = lbm_batch_sync(h->self_batch);
        if (rb != LBM_OK) return rb;
        drop_self_batch(h);
    }
    cudaEvent_t ev = nullptr;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
    cudaEventDestroy(ev);  // released once recorded work completes
    if (e != cudaSuccess) return cuda_fail(e, "lbm_set_stream");
    h->stream = s;
    return LBM_OK;
}

extern "C" int lbm_sync(lbm_t h) {
    if (!h) return fail(LBM_EINVAL, "lbm_sync: NULL handle");
    return sync_status(h);
}

// ---------------------------------------------------------------------------
// Checkpoints.

extern "C" size_t lbm_state_bytes(lbm_t h) {
    return h ? 9 * (size_t)h->nx * h->ny * elem_bytes(h->storage) : 0;
}

extern "C" int lbm_get_state(lbm_t h, void *dst_host, long long *t) {
    if (!h || !dst_host) return fail(LBM_EINVAL, "lbm_get_state: NULL argument");
    size_t row = (size_t)h->nx * h->ny * elem_bytes(h->storage);
    size_t pitch = h->P * elem_bytes(h->storage);
    CK(cudaMemcpy2DAsync(dst_host, row, h->buf[h->cur], pitch, row, 9, cudaMemcpyDeviceToHost,
                         h->stream));
    int rs = sync_status(h);
    if (t) *t = h->t;
    return rs;
}

extern "C" int lbm_set_state(lbm_t h, const void *src_host, long long t) {
    if (!h || !src_host || t < 0) return fail(LBM_EINVAL, "lbm_set_state: bad argument");
    size_t row = (size_t)h->nx * h->ny * elem_bytes(h->storage);
    size_t pitch = h->P * elem_bytes(h->storage);
    CK(cudaMemcpy2DAsync(h->buf[0], pitch, src_host, row, row, 9, cudaMemcpyHostToDevice,
                         h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->cur = 0;
    h->t = t;
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Tile configuration and autotuner.

extern "C" int lbm_set_config(lbm_t h, int vec, int rows, int warps) {
    if (!h) return fail(LBM_EINVAL, "lbm_set_config: NULL handle");
    if (!valid_vec(h->storage, h->nx, vec))
        return fail(LBM_EINVAL, "lbm_set_config: vec must be 1, 2, 4 (or 8 for 16-bit) and divide nx");
    if (rows < 1 || rows > 4096) return fail(LBM_EINVAL, "lbm_set_config: rows in [1, 4096]");
    if (h->a15f && vec == 8) return fail(LBM_EINVAL, "lbm_set_config: c2 fields use vec <= 4");
    if (h->rounding && vec == 8 && warps != 4)
        return fail(LBM_EINVAL, "lbm_set_config: stochastic rounding at vec 8 needs 4 warps");
    if (warps != 1 && warps != 2 && warps != 4 && warps != 8)
        return fail(LBM_EINVAL, "lbm_set_config: warps in {1, 2, 4, 8}");
    if (h->cfg.vec != vec || h->cfg.rows != rows || h->cfg.warps != warps) {
        CK(cudaStreamSynchronize(h->stream));
        drop_graphs(h);
        drop_self_batch(h);
    }
    h->cfg.vec = vec;
    h->cfg.rows = rows;
    h->cfg.warps = warps;
    h->cfg.fit_rows = false;
    CK(prepare_step(h->storage, h->cfg));
    return LBM_OK;
}

extern "C" int lbm_set_pipeline(lbm_t h, int stages) {
    if (!h) return fail(LBM_EINVAL, "lbm_set_pipeline: NULL handle");
    if (stages < 0 || stages > 4)
        return fail(LBM_EINVAL, "lbm_set_pipeline: stages must be 0..4");
    if ((h->rounding || h->a15f) && stages >= 2)
        return fail(LBM_EINVAL, "lbm_set_pipeline: stochastic rounding and c2 fields use the register walk");
    if (h->cfg.stages != stages) {
        CK(cudaStreamSynchronize(h->stream));
        drop_graphs(h);
    }
    h->cfg.stages = stages;
    CK(prepare_step(h->storage, h->cfg));
    return LBM_OK;
}

extern "C" int lbm_set_c2_field(lbm_t h, const double *c2, int on_device) {
    if (!h) return fail(LBM_EINVAL, "lbm_set_c2_field: NULL handle");
    CK(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    drop_self_batch(h);
    if (!c2) {
        if (h->a15f) cudaFree(h->a15f);
        h->a15f = nullptr;
        return LBM_OK;
    }
    if (h->rounding) return fail(LBM_EINVAL, "lbm_set_c2_field: needs nearest rounding");
    if (h->grad != LBM_GRAD_CENTRAL)
        return fail(LBM_EINVAL, "lbm_set_c2_field: needs the central-difference gradient");
    size_t n = (size_t)h->nx * h->ny;
    if (!on_device) {
        for (size_t s = 0; s < n; ++s)
            if (!(c2[s] > 0.0) || !isfinite(c2[s]))
                return fail(LBM_EINVAL, "lbm_set_c2_field: need c2 > 0 at every site");
    }
    if (h->cfg.vec == 8) {  // the field walks use vec <= 4: 4 with a row prefetched
        h->cfg.vec = 4;
        h->cfg.stages = 1;
    }
    if (h->cfg.stages >= 2) h->cfg.stages = 0;
    if (!h->a15f) CK(cudaMalloc(&h->a15f, n * sizeof(float)));
    std::vector<double *> owned;
    double *d = nullptr;
    int rc = stage_field(h, c2, on_device, h->stream, &d, owned);
    if (rc == LBM_OK) {
        cudaError_t e = launch_a15_from_c2(d, h->a15f, (long long)n, h->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "lbm_set_c2_field kernel");
    }
    for (double *p : owned) cudaFreeAsync(p, h->stream);
    if (rc != LBM_OK) return rc;
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

extern "C" int lbm_set_drive(lbm_t h, int on, double amplitude, double period) {
    if (!h) return fail(LBM_EINVAL, "lbm_set_drive: NULL handle");
    if (on) {
        if (h->slab) return fail(LBM_EINVAL, "lbm_set_drive: a slab cannot be driven");
        if (h->nx < 4) return fail(LBM_EINVAL, "lbm_set_drive: needs nx >= 4");
        if (!(period > 0.0) || !isfinite(period))
            return fail(LBM_EINVAL, "lbm_set_drive: period must be finite and > 0");
        if (!isfinite(amplitude) || !(fabs(amplitude) < 1.0))
            return fail(LBM_EINVAL, "lbm_set_drive: need |amplitude| < 1");
    }
    CK(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    drop_self_batch(h);
    h->drive = on != 0;
    h->drive_amp = on ? amplitude : 0.0;
    h->drive_period = on ? period : 0.0;
    return LBM_OK;
}

extern "C" int lbm_set_rounding(lbm_t h, int mode) {
    if (!h) return fail(LBM_EINVAL, "lbm_set_rounding: NULL handle");
    if (mode != LBM_ROUND_NEAREST && mode != LBM_ROUND_STOCHASTIC)
        return fail(LBM_EINVAL, "lbm_set_rounding: unknown mode");
    if (mode == LBM_ROUND_STOCHASTIC && h->storage == ST_F32)
        return fail(LBM_EINVAL, "lbm_set_rounding: stochastic rounding needs 16-bit storage");
    if (mode == LBM_ROUND_STOCHASTIC && h->a15f)
        return fail(LBM_EINVAL, "lbm_set_rounding: not with a c2 field");
    CK(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    drop_self_batch(h);
    h->rounding = mode;
    if (mode == LBM_ROUND_STOCHASTIC) {
        // Stochastic rounding runs on the register walks with vec <= 4 and on
        // the shared-memory row walk at vec 8 with 4 warps per block; other
        // vec-8 configurations move to 4 sites with a row prefetched.
        if (h->cfg.vec == 8 && h->cfg.warps != 4) {
            h->cfg.vec = 4;
            h->cfg.stages = 1;
        }
        if (h->cfg.stages >= 2) h->cfg.stages = 0;
    }
    CK(prepare_step(h->storage, h->cfg));
    return LBM_OK;
}

extern "C" int lbm_set_gradient(lbm_t h, int mode) {
    if (!h) return fail(LBM_EINVAL, "lbm_set_gradient: NULL handle");
    if (mode != LBM_GRAD_CENTRAL && mode != LBM_GRAD_FORWARD)
        return fail(LBM_EINVAL, "lbm_set_gradient: unknown mode");
    if (mode == LBM_GRAD_FORWARD) {
        if (h->storage != ST_F32)
            return fail(LBM_EINVAL, "lbm_set_gradient: the forward difference needs FP32 storage");
        if (h->a15f) return fail(LBM_EINVAL, "lbm_set_gradient: not with a c2 field");
        if (h->slab) return fail(LBM_EINVAL, "lbm_set_gradient: not on a slab");
    }
    CK(cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    drop_self_batch(h);
    h->grad = mode;
    return LBM_OK;
}

extern "C" int lbm_get_gradient(lbm_t h, int *mode) {
    if (!h || !mode) return fail(LBM_EINVAL, "lbm_get_gradient: NULL argument");
    *mode = h->grad;
    return LBM_OK;
}

extern "C" int lbm_get_rounding(lbm_t h, int *mode) {
    if (!h || !mode) return fail(LBM_EINVAL, "lbm_get_rounding: NULL argument");
    *mode = h->rounding;
    return LBM_OK;
}

extern "C" int lbm_get_pipeline(lbm_t h, int *stages, int *active) {
    if (!h) return fail(LBM_EINVAL, "lbm_get_pipeline: NULL handle");
    if (stages) *stages = h->cfg.stages;
    if (active)
        *active = (uses_tma(h->storage, h->cfg) || uses_prefetch(h->storage, h->cfg)) ? 1 : 0;
    return LBM_OK;
}

extern "C" int lbm_get_config(lbm_t h, int *vec, int *rows, int *warps) {
    if (!h) return fail(LBM_EINVAL, "lbm_get_config: NULL handle");
    if (vec) *vec = h->cfg.vec;
    if (rows) *rows = h->cfg.rows;
    if (warps) *warps = h->cfg.warps;
    return LBM_OK;
}

static std::string tune_key(const lbm_grid *h) {
    cudaDeviceProp p;
    std::string dev = "dev";
    if (cudaGetDeviceProperties(&p, h->device) == cudaSuccess) dev = p.name;
    std::ostringstream k;
    k << dev << "|s" << h->storage << "|" << h->nx << "x" << h->ny;
    return k.str();
}

// The cache file is a flat JSON object {"key": [vec, rows, warps, stages], ...}.
static std::map<std::string, TileCfg> read_cache(const char *path) {
    std::map<std::string, TileCfg> m;
    std::ifstream in(path);
    if (!in) return m;
    std::stringstream ss;
    ss << in.rdbuf();
    std::string s = ss.str();
    size_t pos = 0;
    while ((pos = s.find('"', pos)) != std::string::npos) {
        size_t end = s.find('"', pos + 1);
        if (end == std::string::npos) break;
        std::string key = s.substr(pos + 1, end - pos - 1);
        size_t lb = s.find('[', end), rb = s.find(']', end);
        if (lb == std::string::npos || rb == std::string::npos) break;
        TileCfg c;
        if (sscanf(s.c_str() + lb, "[%d , %d , %d , %d]", &c.vec, &c.rows, &c.warps, &c.stages) ==
                4 ||
            sscanf(s.c_str() + lb, "[%d,%d,%d,%d]", &c.vec, &c.rows, &c.warps, &c.stages) == 4)
            m[key] = c;
        pos = rb + 1;
    }
    return m;
}

static void write_cache(const char *path, const std::map<std::string, TileCfg> &m) {
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t k = 0;
    for (auto &kv : m) {
        fprintf(f, "  \"%s\": [%d, %d, %d, %d]%s\n", kv.first.c_str(), kv.second.vec,
                kv.second.rows, kv.second.warps, kv.second.stages, (++k < m.size()) ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

// Times one configuration: `reps` launches from buf[cur] into the other buffer
// (the state itself is not changed).
static int time_cfg(lbm_grid *h, const TileCfg &c, int reps, float *ms_out) {
    TileCfg saved = h->cfg;
    h->cfg = c;
    h->cfg.fit_rows = false;  // time the candidate's own tile height
    cudaError_t e = prepare_step(h->storage, c);
    if (e == cudaSuccess) e = launch_one(h, h->cur);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(h->ev[0], h->stream);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_one(h, h->cur);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev[1], h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(h->ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
    h->cfg = saved;
    if (e != cudaSuccess) return cuda_fail(e, "lbm_tune");
    *ms_out = ms / reps;
    return LBM_OK;
}

extern "C" int lbm_tune(lbm_t h, const char *cache_path) {
    if (!h) return fail(LBM_EINVAL, "lbm_tune: NULL handle");
    std::string key = tune_key(h);
    std::map<std::string, TileCfg> cache;
    if (cache_path) {
        cache = read_cache(cache_path);
        auto it = cache.find(key);
        if (it != cache.end() && valid_vec(h->storage, h->nx, it->second.vec)) {
            int rc = lbm_set_config(h, it->second.vec, it->second.rows, it->second.warps);
            if (rc != LBM_OK) return rc;
            return lbm_set_pipeline(h, it->second.stages);
        }
    }
    CK(cudaStreamSynchronize(h->stream));
    long long sites = (long long)h->nx * h->ny;
    int reps = (int)std::max<long long>(3, std::min<long long>(50, 200000000LL / (sites + 1)));
    TileCfg best = h->cfg;
    float best_ms = 1e30f;
    const int vecs[] = {1, 2, 4, 8};
    const int rowss[] = {4, 8, 16, 32, 64, 128};
    const int warpss[] = {2, 4, 8};
    for (int v : vecs) {
        if (!valid_vec(h->storage, h->nx, v)) continue;
        if ((h->rounding || h->a15f) && v == 8) continue;
        for (int r : rowss) {
            if (r > 2 * h->ny && r != 4) continue;
            for (int w : warpss) {
                const bool tma_ok = v == tma_vec(h->storage);
                const bool pf_ok =
                    v == prefetch_vec(h->storage) || (h->storage != ST_F32 && v == 8);
                for (int nst = 0; nst <= 4; ++nst) {
                    if (nst == 1 && !pf_ok) continue;
                    if (nst >= 2 && (!tma_ok || h->rounding || h->a15f)) continue;
                    TileCfg c;
                    c.vec = v;
                    c.rows = r;
                    c.warps = w;
                    c.stages = nst;
                    float ms;
                    int rc = time_cfg(h, c, reps, &ms);
                    if (rc != LBM_OK) return rc;
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = c;
                    }
                }
            }
        }
    }
    int rc = lbm_set_config(h, best.vec, best.rows, best.warps);
    if (rc == LBM_OK) rc = lbm_set_pipeline(h, best.stages);
    if (rc != LBM_OK) return rc;
    if (cache_path) {
        cache[key] = best;
        write_cache(cache_path, cache);
    }
    return LBM_OK;
}
