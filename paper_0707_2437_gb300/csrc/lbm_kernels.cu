// Kernels of liblbm.so: the fused step, equilibrium initialisation, moments,
// and the FP64 reductions (grid totals and Fourier coefficients).
#include <math.h>

#include <mutex>
#include <vector>

#include "lbm_internal.h"

namespace vss {

// The FP32 constants are chosen so that the linear part of the collision
// conserves the density and momentum deviations exactly (with the weights of
// lbm_device.cuh): om + om1 == 1 in FP32 (the one of them in [0.5, 2] is
// rounded, the other is 1 minus it, which is exact there), and the momentum
// coefficient (1/tau)/T is carried as a rounded value plus its remainder.
Coef make_coef(double tau, double c2, double rho0) {
    Coef c;
    float om = (float)(1.0 / tau);
    float om1;
    if (om >= 0.5f) {
        om1 = 1.0f - om;  // exact: om in [0.5, 2) for tau in (0.5, 2]
    } else {
        om1 = (float)(1.0 - 1.0 / tau);  // in (0.5, 1)
        om = 1.0f - om1;                  // exact
    }
    c.om = om;
    c.om1 = om1;
    const double w3 = (double)om / VSS_T_D;
    c.w3 = (float)w3;
    c.w3lo = (float)(w3 - (double)c.w3);
    c.w45 = (float)(4.5 * (double)om);
    c.a15 = a15_of_alpha(1.0 / 3.0 - c2);  // Section 3, Eq. 8 with c_1^2 = 1/3
    c.rho0 = (float)rho0;
    return c;
}

bool valid_vec(int storage, int nx, int vec) {
    if (vec != 1 && vec != 2 && vec != 4 && vec != 8) return false;
    if (vec == 8 && storage == ST_F32) return false;
    return nx % vec == 0;
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  The single-grid step kernels are launched
// with programmatic stream serialization allowed: each block first lets the next launch on the stream
// start (the next grid is launched once every block of this one has started
// or exited, so its blocks only take SM slots this grid no longer needs), then
// waits until the previous grid has completed and its memory is visible, and
// only then touches global memory.  The next step's launch latency is thereby
// hidden behind this step's tail.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block,
                              size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// Fused step: one warp per (strip, row segment) tile.

template <int S, int V, bool PF, int RND = 0, int VA = 0, int GR = 0>
__global__ void __launch_bounds__(256, 2)
    k_step(const void *__restrict__ fin, void *__restrict__ fout, int nx, int ny, size_t P,
           int nstrips, long long ntiles, int rows, Coef c, const uint32_t *tdev,
           uint32_t toff, const float *__restrict__ a15f) {
    pdl_enter();
    long long tile = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (tile >= ntiles) return;  // whole warps leave together
    int strip = (int)(tile % nstrips);
    int seg = (int)(tile / nstrips);
    int x0 = strip * 32 * V;
    int y0 = seg * rows;
    int y1 = min(ny, y0 + rows);
    Walker<S, V, LD_NC, RND, VA, 32, GR> w(fin, fout, nx, ny, P, x0);
    if constexpr (VA) w.a15f = a15f;
    // Stochastic rounding is seeded by the step being computed: a device
    // counter (set before each graph replay) plus this launch's offset.
    if constexpr (RND) w.set_step((tdev ? *tdev : 0u) + toff);
    // Neighbouring segments walk in opposite directions so that the two rows
    // they share are read by both at about the same time.
    if constexpr (PF)
        w.run_prefetch(y0, y1, (seg & 1) ? -1 : 1, c);
    else
        w.run(y0, y1, (seg & 1) ? -1 : 1, c);
}

// Wide prefetching walk for the 16-bit kinds: 8 sites per lane (128-bit
// loads) with one row prefetched; three rows of 8 sites need more than 128
// registers, so this kernel runs one 8-warp block per SM (up to 255 registers).
template <int S>
__global__ void __launch_bounds__(256, 1)
    k_step_wide(const void *__restrict__ fin, void *__restrict__ fout, int nx, int ny, size_t P,
                int nstrips, long long ntiles, int rows, Coef c) {
    pdl_enter();
    long long tile = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (tile >= ntiles) return;
    int strip = (int)(tile % nstrips);
    int seg = (int)(tile / nstrips);
    int x0 = strip * 32 * 8;
    int y0 = seg * rows;
    int y1 = min(ny, y0 + rows);
    Walker<S, 8> w(fin, fout, nx, ny, P, x0);
    w.run_prefetch(y0, y1, (seg & 1) ? -1 : 1, c);
}

// The 8-site 16-bit walk of the batch kernels in the step kernel: rows move
// through shared memory with cp.async (a landing slot and a stash per warp,
// 36.9 KB per block of 4 warps), one row in flight while the warp computes.
// The default for 16-bit grids whose nx is a multiple of 8 and that have
// enough tiles (see default_cfg), with either rounding.
template <int S, int RND>
__global__ void __launch_bounds__(128, 4)
    k_step_async(const void *__restrict__ fin, void *__restrict__ fout, int nx, int ny, size_t P,
                 int nstrips, long long ntiles, int rows, Coef c, const uint32_t *tdev,
                 uint32_t toff) {
    __shared__ uint4 rowbuf[4][2 * 9 * 32];
    pdl_enter();
    long long tile = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (tile >= ntiles) return;
    int strip = (int)(tile % nstrips);
    int seg = (int)(tile / nstrips);
    int x0 = strip * 32 * 8;
    int y0 = seg * rows;
    int y1 = min(ny, y0 + rows);
    Walker<S, 8, LD_NC, RND> w(fin, fout, nx, ny, P, x0);
    if constexpr (RND) w.set_step((tdev ? *tdev : 0u) + toff);
    w.run_async(y0, y1, (seg & 1) ? -1 : 1, c, &rowbuf[threadIdx.x >> 5][0]);
}

// Bulk-copy pipeline variant: one warp per tile, NST shared-memory stages per
// warp (dynamic shared memory: barriers first, then the stages).
constexpr unsigned long long kWaitLimitNs = 1000000000ULL;  // 1 s per wait

template <int S, int NST>
__global__ void __launch_bounds__(256, 2)
    k_step_tma(const void *__restrict__ fin, void *__restrict__ fout, int nx, int ny, size_t P,
               int nstrips, long long ntiles, int rows, Coef c, int *status) {
    pdl_enter();
    extern __shared__ __align__(128) unsigned char smem[];
    const int nwb = blockDim.x >> 5;
    const int wib = threadIdx.x >> 5;
    long long tile = (long long)blockIdx.x * nwb + wib;
    if (tile >= ntiles) return;
    constexpr int V = TmaGeom<S>::V;
    int strip = (int)(tile % nstrips);
    int seg = (int)(tile / nstrips);
    int x0 = strip * 32 * V;
    int y0 = seg * rows;
    int y1 = min(ny, y0 + rows);
    uint32_t bars = smem_u32(smem) + (uint32_t)(wib * NST * 8);
    unsigned char *st = smem + tma_bar_bytes(nwb, NST) + (size_t)wib * NST * TmaGeom<S>::STAGE_B;
    TmaWalker<S, NST> w(fin, fout, nx, ny, P, x0, st, bars, kWaitLimitNs);
    w.run(y0, y1, (seg & 1) ? -1 : 1, c, status);
}

// Resident warps of a step kernel with blocks of `warps` warps on the
// current device, found once per kernel, block size and device.
static long long resident_warps(const void *fn, int warps) {
    struct Entry {
        const void *fn;
        int warps, dev;
        long long w;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (const Entry &e : cache)
            if (e.fn == fn && e.warps == warps && e.dev == dev) return e.w;
    }
    int blocks = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, 32 * warps, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    const long long w = (long long)blocks * warps * sms;
    std::lock_guard<std::mutex> lk(mu);
    cache.push_back(Entry{fn, warps, dev, w});
    return w;
}

// Tile height of a register-walk launch in the default configuration.  Each
// warp walks its tile's rows one after another, so a grid with fewer tiles
// than resident warps leaves warps idle and its step takes a whole tile
// walk however small the grid, and a grid whose tiles need between one and
// two waves runs its second wave partly empty.  So, with the configured
// height r0 (16):
//   tiles at r0 >= 2 waves        -> r0;
//   between one and two waves     -> the lowest height up to 2 r0 at which
//                                    one wave holds every tile (else r0);
//   at least 3/4 of one wave      -> r0;
//   fewer                         -> the lowest height down to 2 at which the
//                                    tiles still fit one wave (more, shorter
//                                    tiles; the extra rows each pulls come
//                                    mostly from L2).
// Measured on 2048^2: the FP32 c2-field walk (2-site, 4096 tiles at 16 rows)
// 63.2 -> 58.9 us per launch at 27 rows; 1024^2 FP32 and FP16-delta steps
// took a whole 16-row walk (31 and 25 us per launch for 512 tiles).
static TileCfg fit_tile(const TileCfg &cfg, const void *fn, int nx, int ny) {
    if (!cfg.fit_rows) return cfg;
    const long long wave = resident_warps(fn, cfg.warps);
    if (wave <= 0) return cfg;
    const long long nstrips = (nx + 32LL * cfg.vec - 1) / (32LL * cfg.vec);
    auto tiles = [&](int r) { return nstrips * ((ny + r - 1) / r); };
    const int r0 = cfg.rows;
    TileCfg c = cfg;
    const long long t0 = tiles(r0);
    if (t0 >= 2 * wave || 4 * t0 >= 3 * wave && t0 <= wave) return c;
    if (t0 > wave) {
        for (int r = r0 + 1; r <= 2 * r0; ++r)
            if (tiles(r) <= wave) {
                c.rows = r;
                return c;
            }
        return c;
    }
    int r = r0;
    while (r > 2 && tiles(r - 1) <= wave) --r;
    c.rows = r;
    return c;
}

template <int S, int V, int RND>
static Err launch_step_t(const TileCfg &cfg, const void *fin, void *fout, int nx, int ny, size_t P,
                         const Coef &c, const uint32_t *tdev, uint32_t toff, const float *a15f,
                         cudaStream_t st) {
    // Launches `kernel` over the grid's tiles at the fitted tile height.
    auto go = [&](auto kernel, auto... extra) -> Err {
        const TileCfg t = fit_tile(cfg, (const void *)kernel, nx, ny);
        const StepGeom g = step_geom(nx, ny, t);
        const unsigned nb = (unsigned)((g.ntiles + t.warps - 1) / t.warps);
        return launch_pdl(kernel, nb, 32u * t.warps, 0, st, fin, fout, nx, ny, P, g.nstrips,
                          g.ntiles, t.rows, c, extra...);
    };
    if (a15f) {
        // Spatially varying alpha: the register walks (prefetching at 64-bit
        // vectors for 16-bit storage), nearest rounding.
        if constexpr (RND == 0 && V <= 4) {
            if (uses_prefetch(S, cfg)) {
                if constexpr (Pack<S, V>::BYTES == 8)
                    return go(k_step<S, V, true, 0, 1>, tdev, toff, a15f);
                else
                    return cudaErrorInvalidValue;
            } else if constexpr (S == ST_F32 && V == 4) {
                return cudaErrorInvalidValue;  // launch_step_s runs the 2-site walk instead
            } else {
                return go(k_step<S, V, false, 0, 1>, tdev, toff, a15f);
            }
        } else {
            return cudaErrorInvalidValue;
        }
    }
    if (V == 8 && cfg.warps == 4 && (RND || !uses_prefetch(S, cfg))) {
        // The shared-memory row walk (stochastic rounding: also in place of
        // the register prefetch, which has no rounding variant at 8 sites).
        if constexpr (S != ST_F32 && V == 8)
            return go(k_step_async<S, RND>, tdev, toff);
        else
            return cudaErrorInvalidValue;
    } else if (uses_prefetch(S, cfg) && V == 8) {
        if constexpr (S != ST_F32 && V == 8 && RND == 0)
            return go(k_step_wide<S>);
        else
            return cudaErrorInvalidValue;
    } else if (uses_prefetch(S, cfg)) {
        if constexpr (Pack<S, V>::BYTES == 8)
            return go(k_step<S, V, true, RND>, tdev, toff, (const float *)nullptr);
        else
            return cudaErrorInvalidValue;
    } else {
        return go(k_step<S, V, false, RND>, tdev, toff, (const float *)nullptr);
    }
}

template <int S, int NST>
static Err launch_tma_t(const TileCfg &cfg, const void *fin, void *fout, int nx, int ny, size_t P,
                        const Coef &c, int *status, cudaStream_t st) {
    StepGeom g = step_geom(nx, ny, cfg);
    long long blocks = (g.ntiles + cfg.warps - 1) / cfg.warps;
    int smem = tma_smem_bytes<S>(cfg.warps, NST);
    return launch_pdl(k_step_tma<S, NST>, (unsigned)blocks, 32u * cfg.warps, (size_t)smem, st, fin,
                      fout, nx, ny, P, g.nstrips, g.ntiles, cfg.rows, c, status);
}

template <int S, int NST>
static Err prepare_tma_t() {
    // Enough dynamic shared memory for the largest block (8 warps).
    return cudaFuncSetAttribute(k_step_tma<S, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                tma_smem_bytes<S>(8, NST));
}

template <int S>
static Err prepare_s(int stages) {
    switch (stages) {
        case 2:
            return prepare_tma_t<S, 2>();
        case 3:
            return prepare_tma_t<S, 3>();
        case 4:
            return prepare_tma_t<S, 4>();
        default:
            return cudaErrorInvalidValue;
    }
}

Err prepare_step(int storage, const TileCfg &cfg) {
    if (!uses_tma(storage, cfg)) return cudaSuccess;
    if (tma_smem_bytes<ST_F32>(cfg.warps, cfg.stages) > 227 * 1024) return cudaErrorInvalidValue;
    switch (storage) {
        case ST_F32:
            return prepare_s<ST_F32>(cfg.stages);
        case ST_F16:
            return prepare_s<ST_F16>(cfg.stages);
        case ST_BF16:
            return prepare_s<ST_BF16>(cfg.stages);
        default:
            return cudaErrorInvalidValue;
    }
}

template <int S>
static Err launch_step_s(const TileCfg &cfg, const void *fin, void *fout, int nx, int ny, size_t P,
                         const Coef &c, int *status, int rnd, const uint32_t *tdev,
                         uint32_t toff, const float *a15f, cudaStream_t st) {
    if (a15f && (rnd || cfg.vec == 8)) return cudaErrorInvalidValue;
    if (S == ST_F32 && a15f && cfg.vec == 4) {
        // FP32 with a c2 field: the 4-site walk needs more than 128 registers
        // with the field's four alphas (it spilled 60 bytes); the 2-site walk
        // with one row of loads prefetched runs at the same speed within 120.
        TileCfg c2 = cfg;
        c2.vec = 2;
        c2.stages = 1;
        return launch_step_t<S, 2, 0>(c2, fin, fout, nx, ny, P, c, tdev, toff, a15f, st);
    }
    if (rnd) {
        // Stochastic rounding: register walks with vec 1, 2 or 4, and the
        // shared-memory row walk at vec 8 (4 warps per block).
        if constexpr (S == ST_F32) {
            return cudaErrorInvalidValue;
        } else {
            switch (cfg.vec) {
                case 8:
                    return launch_step_t<S, 8, 1>(cfg, fin, fout, nx, ny, P, c, tdev, toff, nullptr, st);
                case 1:
                    return launch_step_t<S, 1, 1>(cfg, fin, fout, nx, ny, P, c, tdev, toff, nullptr, st);
                case 2:
                    return launch_step_t<S, 2, 1>(cfg, fin, fout, nx, ny, P, c, tdev, toff, nullptr, st);
                case 4:
                    return launch_step_t<S, 4, 1>(cfg, fin, fout, nx, ny, P, c, tdev, toff, nullptr, st);
                default:
                    return cudaErrorInvalidValue;
            }
        }
    }
    if (uses_tma(S, cfg) && !a15f) {
        switch (cfg.stages) {
            case 2:
                return launch_tma_t<S, 2>(cfg, fin, fout, nx, ny, P, c, status, st);
            case 3:
                return launch_tma_t<S, 3>(cfg, fin, fout, nx, ny, P, c, status, st);
            case 4:
                return launch_tma_t<S, 4>(cfg, fin, fout, nx, ny, P, c, status, st);
            default:
                return cudaErrorInvalidValue;
        }
    }
    switch (cfg.vec) {
        case 1:
            return launch_step_t<S, 1, 0>(cfg, fin, fout, nx, ny, P, c, tdev, toff, a15f, st);
        case 2:
            return launch_step_t<S, 2, 0>(cfg, fin, fout, nx, ny, P, c, tdev, toff, a15f, st);
        case 4:
            return launch_step_t<S, 4, 0>(cfg, fin, fout, nx, ny, P, c, tdev, toff, a15f, st);
        case 8:
            if constexpr (S != ST_F32)
                return launch_step_t<S, 8, 0>(cfg, fin, fout, nx, ny, P, c, tdev, toff, a15f, st);
            return cudaErrorInvalidValue;
        default:
            return cudaErrorInvalidValue;
    }
}

Err launch_step_forward(const TileCfg &cfg, const void *fin, void *fout, int nx, int ny, size_t P,
                        const Coef &c, cudaStream_t st) {
    // One site per lane (any nx), the configured tile height and block size.
    TileCfg c1 = cfg;
    c1.vec = 1;
    c1.stages = 0;
    c1 = fit_tile(c1, (const void *)k_step<ST_F32, 1, false, 0, 0, 1>, nx, ny);
    StepGeom g = step_geom(nx, ny, c1);
    long long blocks = (g.ntiles + c1.warps - 1) / c1.warps;
    return launch_pdl(k_step<ST_F32, 1, false, 0, 0, 1>, (unsigned)blocks, 32u * c1.warps, 0, st,
                      fin, fout, nx, ny, P, g.nstrips, g.ntiles, c1.rows, c,
                      (const uint32_t *)nullptr, 0u, (const float *)nullptr);
}

Err launch_step(int storage, const TileCfg &cfg, const void *fin, void *fout, int nx, int ny,
                size_t P, const Coef &c, int *status, int rnd, const uint32_t *tdev, uint32_t toff,
                const float *a15f, cudaStream_t st) {
    switch (storage) {
        case ST_F32:
            return launch_step_s<ST_F32>(cfg, fin, fout, nx, ny, P, c, status, rnd, tdev, toff,
                                         a15f, st);
        case ST_F16:
            return launch_step_s<ST_F16>(cfg, fin, fout, nx, ny, P, c, status, rnd, tdev, toff,
                                         a15f, st);
        case ST_BF16:
            return launch_step_s<ST_BF16>(cfg, fin, fout, nx, ny, P, c, status, rnd, tdev, toff,
                                          a15f, st);
        default:
            return cudaErrorInvalidValue;
    }
}

__global__ void k_set_u32(uint32_t *p, uint32_t v) { *p = v; }

// 1.5 alpha per site from c^2 per site (alpha = 1/3 - c^2, Section 3, Eq. 8).
__global__ void k_a15_from_c2(const double *c2, float *a15, long long n) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x)
        a15[s] = a15_of_alpha(1.0 / 3.0 - c2[s]);
}

Err launch_a15_from_c2(const double *c2, float *a15, long long n, cudaStream_t st) {
    long long b = (n + 255) / 256;
    k_a15_from_c2<<<(unsigned)(b < 4096 ? b : 4096), 256, 0, st>>>(c2, a15, n);
    return cudaGetLastError();
}

Err launch_set_u32(uint32_t *p, uint32_t v, cudaStream_t st) {
    k_set_u32<<<1, 1, 0, st>>>(p, v);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Element conversions from / to double (not on the hot path).

template <int S>
__device__ __forceinline__ double ld_elem_d(const void *f, size_t idx) {
    if constexpr (S == ST_F32)
        return (double)reinterpret_cast<const float *>(f)[idx];
    else if constexpr (S == ST_F16)
        return (double)__half2float(reinterpret_cast<const __half *>(f)[idx]);
    else
        return (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(f)[idx]);
}

template <int S>
__device__ __forceinline__ void st_elem_d(void *f, size_t idx, double v) {
    if constexpr (S == ST_F32)
        reinterpret_cast<float *>(f)[idx] = (float)v;
    else if constexpr (S == ST_F16)
        reinterpret_cast<__half *>(f)[idx] = __double2half(v);
    else
        reinterpret_cast<__nv_bfloat16 *>(f)[idx] = __double2bfloat16(v);
}

__device__ __forceinline__ int wrapi(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// Weights and links in double for the FP64 side kernels.
__device__ __forceinline__ double wd(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}

template <int S>
__device__ __forceinline__ float ld_elem_f(const void *f, size_t idx) {
    if constexpr (S == ST_F32)
        return reinterpret_cast<const float *>(f)[idx];
    else if constexpr (S == ST_F16)
        return __half2float(reinterpret_cast<const __half *>(f)[idx]);
    else
        return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(f)[idx]);
}

template <int S>
__device__ __forceinline__ void st_elem_f(void *f, size_t idx, float v) {
    if constexpr (S == ST_F32)
        reinterpret_cast<float *>(f)[idx] = v;
    else if constexpr (S == ST_F16)
        reinterpret_cast<__half *>(f)[idx] = __float2half_rn(v);
    else
        reinterpret_cast<__nv_bfloat16 *>(f)[idx] = __float2bfloat16_rn(v);
}

// Equilibrium initialisation (Section 2, Eq. 2).  Each site computes the
// equilibrium of its own fields in FP32, as h_i = (fbar_i - w_i rho0)/w_i =
// drho + rho (3 e.u + 9/2 (e.u)^2 - 3/2 u.u), and writes direction i where
// the pull of that site will find it: plane i at x - e_i.  Only the deviation
// drho = rho - rho0 is formed in FP64 (it can be far below FP32's resolution
// of rho near 1).
template <int S>
__global__ void k_init(void *f, int nx, int ny, size_t P, double rho0, const double *rho,
                       const double *ux, const double *uy) {
    long long n = (long long)nx * ny;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(s % nx), y = (int)(s / nx);
        const double r = rho[s];
        const float dr = (float)(r - rho0);
        const float rf = (float)r;
        const float u = (float)ux[s], v = (float)uy[s];
        const float m15usq = -1.5f * __fmaf_rn(u, u, __fmul_rn(v, v));
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float eu = EXi(i) * u + EYi(i) * v;  // e components are 0 and +-1
            const float poly = __fmaf_rn(__fmul_rn(4.5f, eu), eu, __fmaf_rn(3.0f, eu, m15usq));
            const size_t dst = (size_t)wrapi(y - EYi(i), ny) * nx + wrapi(x - EXi(i), nx);
            st_elem_f<S>(f, (size_t)i * P + dst, __fmaf_rn(rf, poly, dr));
        }
    }
}

// Driven channel of Section 4 (the runs of Fig. 1), applied after a step to
// the buffer the step wrote (post-collision values stored at their source
// site): column 0 becomes the equilibrium at rho = 1 + amp sin(2 pi t /
// period), u = 0, and columns nx-2 and nx-1 the equilibrium at rho = 1,
// u = 0.  At u = 0 the equilibrium of Eq. 2 is w_i rho, so the stored
// deviation is h_i = rho - rho0 in every direction.  The step number is
// t = *tdev + toff (tdev may be NULL), taken mod 2^32.
template <int S>
__global__ void k_drive_x(void *f, int nx, int ny, size_t P, double rho0, double amp,
                          double period, const uint32_t *tdev, uint32_t toff) {
    const uint32_t t = (tdev ? *tdev : 0u) + toff;
    const double hb = (1.0 + amp * sin(6.283185307179586476925287 * (double)t / period)) - rho0;
    const double hr = 1.0 - rho0;
    const long long n = 27LL * ny;  // 9 planes x 3 columns x ny rows
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int col = (int)(k % 3);
        const long long r = k / 3;
        const int y = (int)(r % ny), i = (int)(r / ny);
        const int x = col == 0 ? 0 : nx - 3 + col;  // 0, nx-2, nx-1
        st_elem_d<S>(f, (size_t)i * P + (size_t)y * nx + x, col == 0 ? hb : hr);
    }
}

// Moments (Section 2, Eq. 3) of the current state in FP64.
template <int S>
__device__ __forceinline__ void site_moments_d(const void *f, int nx, int ny, size_t P, int x,
                                               int y, double rho0, double &dr, double &jx,
                                               double &jy) {
    dr = 0.0;
    jx = 0.0;
    jy = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        size_t src = (size_t)wrapi(y - EYi(i), ny) * nx + wrapi(x - EXi(i), nx);
        double g = wd(i) * ld_elem_d<S>(f, (size_t)i * P + src);
        dr += g;
        jx += g * EXi(i);
        jy += g * EYi(i);
    }
}

// Moments (Section 2, Eq. 3) of every site, in FP32 arithmetic: drho = sum
// w_i h_i and j = sum w_i h_i e_i of the pulled values, u = j / rho.  The
// outputs are FP64 arrays with rho = rho0 + drho formed in FP64.  (The FP64
// reductions below use FP64 per-site moments: their totals and Fourier
// coefficients carry the accuracy of the mass checks and wave fits.)
template <int S>
__global__ void k_moments(const void *f, int nx, int ny, size_t P, double rho0, double *rho,
                          double *ux, double *uy) {
    long long n = (long long)nx * ny;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(s % nx), y = (int)(s / nx);
        float dr = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const size_t src = (size_t)wrapi(y - EYi(i), ny) * nx + wrapi(x - EXi(i), nx);
            const float wi = i == 0 ? 4.0f / 9.0f : (i < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
            const float g = __fmul_rn(wi, ld_elem_f<S>(f, (size_t)i * P + src));
            dr = __fadd_rn(dr, g);
            if (EXi(i)) jx = EXi(i) > 0 ? __fadd_rn(jx, g) : __fsub_rn(jx, g);
            if (EYi(i)) jy = EYi(i) > 0 ? __fadd_rn(jy, g) : __fsub_rn(jy, g);
        }
        const double r = rho0 + (double)dr;
        const float rf = (float)r;
        if (rho) rho[s] = r;
        if (ux) ux[s] = (double)__fdiv_rn(jx, rf);
        if (uy) uy[s] = (double)__fdiv_rn(jy, rf);
    }
}

// ---------------------------------------------------------------------------
// FP64 reductions in a fixed order: RB blocks of RT threads; thread k of block
// b takes sites b*RT + k, then + RB*RT, ...; each block sums its threads in a
// fixed tree; a second one-block kernel sums the block partials in order.

constexpr int RT = 256;
constexpr int RB_MAX = kReduceBlocksMax;

int reduce_blocks(int nx, int ny) {
    long long n = (long long)nx * ny;
    long long b = (n + RT - 1) / RT;
    return (int)(b < RB_MAX ? b : RB_MAX);
}

template <int K>
__device__ __forceinline__ void block_sum_store(double (&v)[K], double *out_block) {
    __shared__ double sh[K][RT];
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int s = RT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
#pragma unroll
            for (int k = 0; k < K; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) out_block[k] = sh[k][0];
    }
}

template <int K>
__global__ void k_final(const double *partials, int nblocks, double *out) {
    // One block: thread k sums partial k of every block in block order.
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * K + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

template <int S>
__global__ void __launch_bounds__(RT)
    k_sums(const void *f, int nx, int ny, size_t P, double *partials) {
    long long n = (long long)nx * ny;
    double v[3] = {0.0, 0.0, 0.0};
    for (long long s = (long long)blockIdx.x * RT + threadIdx.x; s < n;
         s += (long long)gridDim.x * RT) {
        // Grid totals do not depend on streaming (each plane is permuted), so
        // the stored planes are summed where they lie.
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            double g = wd(i) * ld_elem_d<S>(f, (size_t)i * P + s);
            v[0] += g;
            v[1] += g * EXi(i);
            v[2] += g * EYi(i);
        }
    }
    block_sum_store<3>(v, partials + (size_t)blockIdx.x * 3);
}

template <int S>
__global__ void __launch_bounds__(RT)
    k_mode(const void *f, int nx, int ny, size_t P, double rho0, int field, int kx, int ky,
           double *partials) {
    long long n = (long long)nx * ny;
    double v[2] = {0.0, 0.0};
    for (long long s = (long long)blockIdx.x * RT + threadIdx.x; s < n;
         s += (long long)gridDim.x * RT) {
        int x = (int)(s % nx), y = (int)(s / nx);
        double dr, jx, jy;
        site_moments_d<S>(f, nx, ny, P, x, y, rho0, dr, jx, jy);
        double val = field == 0 ? dr : (field == 1 ? jx / (rho0 + dr) : jy / (rho0 + dr));
        // Phase 2 pi (kx x / nx + ky y / ny), reduced exactly before scaling.
        long long px = ((long long)kx * x) % nx;
        long long py = ((long long)ky * y) % ny;
        double ph = 2.0 * ((double)px / nx + (double)py / ny);
        double sn, cs;
        sincospi(ph, &sn, &cs);
        v[0] += val * cs;
        v[1] += val * sn;
    }
    block_sum_store<2>(v, partials + (size_t)blockIdx.x * 2);
}

__global__ void k_scale2(double *out, double s) {
    if (threadIdx.x < 2) out[threadIdx.x] *= s;
}

// ---------------------------------------------------------------------------
// Launchers.

#define DISPATCH_S(storage, CALL)                  \
    switch (storage) {                             \
        case ST_F32: {                             \
            constexpr int S_ = ST_F32;             \
            CALL;                                  \
        } break;                                   \
        case ST_F16: {                             \
            constexpr int S_ = ST_F16;             \
            CALL;                                  \
        } break;                                   \
        case ST_BF16: {                            \
            constexpr int S_ = ST_BF16;            \
            CALL;                                  \
        } break;                                   \
        default:                                   \
            return cudaErrorInvalidValue;          \
    }

static unsigned side_blocks(int nx, int ny) {
    long long n = (long long)nx * ny;
    long long b = (n + 255) / 256;
    return (unsigned)(b < 4096 ? b : 4096);
}

Err launch_init(int storage, void *f, int nx, int ny, size_t P, double rho0, const double *rho,
                const double *ux, const double *uy, cudaStream_t st) {
    DISPATCH_S(storage, (k_init<S_><<<side_blocks(nx, ny), 256, 0, st>>>(f, nx, ny, P, rho0, rho,
                                                                         ux, uy)));
    return cudaGetLastError();
}

Err launch_drive_x(int storage, void *f, int nx, int ny, size_t P, double rho0, double amp,
                   double period, const uint32_t *tdev, uint32_t toff, cudaStream_t st) {
    long long b = (27LL * ny + 255) / 256;
    unsigned nb = (unsigned)(b < 1024 ? b : 1024);
    DISPATCH_S(storage, (k_drive_x<S_><<<nb, 256, 0, st>>>(f, nx, ny, P, rho0, amp, period, tdev,
                                                            toff)));
    return cudaGetLastError();
}

Err launch_moments(int storage, const void *f, int nx, int ny, size_t P, double rho0, double *rho,
                   double *ux, double *uy, cudaStream_t st) {
    DISPATCH_S(storage, (k_moments<S_><<<side_blocks(nx, ny), 256, 0, st>>>(f, nx, ny, P, rho0,
                                                                            rho, ux, uy)));
    return cudaGetLastError();
}

Err launch_sums(int storage, const void *f, int nx, int ny, size_t P, double *partials,
                double *out3, cudaStream_t st) {
    int nb = reduce_blocks(nx, ny);
    DISPATCH_S(storage, (k_sums<S_><<<nb, RT, 0, st>>>(f, nx, ny, P, partials)));
    k_final<3><<<1, 32, 0, st>>>(partials, nb, out3);
    return cudaGetLastError();
}

Err launch_mode(int storage, const void *f, int nx, int ny, size_t P, double rho0, int field,
                int kx, int ky, double *partials, double *out2, cudaStream_t st) {
    int nb = reduce_blocks(nx, ny);
    DISPATCH_S(storage,
               (k_mode<S_><<<nb, RT, 0, st>>>(f, nx, ny, P, rho0, field, kx, ky, partials)));
    k_final<2><<<1, 32, 0, st>>>(partials, nb, out2);
    k_scale2<<<1, 32, 0, st>>>(out2, 2.0 / ((double)nx * ny));
    return cudaGetLastError();
}

}  // namespace vss

#ifdef VSS_BOUNDS_CHECK
// Debug builds only: the bounds-check record of the step kernels.
extern "C" int lbm_debug_oob(unsigned long long *out2) {
    return cudaMemcpyFromSymbol(out2, vss::vss_oob_record, sizeof(unsigned long long) * 2) ==
                   cudaSuccess
               ? 0
               : -3;
}
#endif
