// Grid totals without any allocation (lbm_sums_noalloc).
//
// For callers that cannot allocate device memory on their own: code running
// inside a custom memory pool or an allocator that forbids outside
// cudaMalloc, code where every byte is budgeted up front, or code that must
// not make an allocating CUDA call at that point.  lbm_sums needs a handle,
// and a handle owns device buffers; this entry point reduces a state buffer
// the caller already holds and keeps its reduction scratch in a fixed array
// in the library's own device memory.
//
// The scratch is a file-scope device array of kSlots doubles (24.1 KiB per
// GPU that loads the library, held until the process exits).  It holds one
// partial triple per reduction block (at most 1024 blocks) and the 3-value
// result.  Every call shares it and leaves its contents behind; no slot is
// read by a call before that call has written it, so nothing needs clearing.
// Calls whose work overlaps on the GPU (on different streams, or from
// different threads without ordering) race on the array and may return wrong
// totals: keep calls on one device ordered.
#include <math.h>

#include <mutex>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace vss;

namespace {

// One partial triple per reduction block: reduce_blocks never returns more
// than kReduceBlocksMax, so the scratch follows that cap.
constexpr int kMaxBlocks = kReduceBlocksMax;
static_assert(kMaxBlocks >= 1, "the reduction needs at least one block");
constexpr int kSlots = 3 * kMaxBlocks + 8;      // partial triples, then the result
static __device__ __align__(256) double g_noalloc_scratch[kSlots];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the array's name in host code is only a stand-in).
int scratch_for_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("lbm_sums_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return LBM_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("lbm_sums_noalloc: device index out of range");
        return LBM_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("lbm_sums_noalloc: cudaGetSymbolAddress: ") +
                      cudaGetErrorString(e));
            return LBM_ECUDA;
        }
        g_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_ptr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_sums_noalloc(const void *f, int nx, int ny, size_t plane_stride, int storage,
                                double rho0, void *cuda_stream, double *out3) {
    if (!f || !out3) {
        set_error("lbm_sums_noalloc: NULL argument");
        return LBM_EINVAL;
    }
    if (nx < 1 || ny < 1 || (long long)nx * ny > 0x7fffffffLL) {
        set_error("lbm_sums_noalloc: need nx, ny >= 1 and nx*ny <= 2^31 - 1 sites");
        return LBM_EINVAL;
    }
    if (plane_stride < (size_t)nx * (size_t)ny) {
        set_error("lbm_sums_noalloc: plane_stride must be at least nx*ny");
        return LBM_EINVAL;
    }
    if (storage < 0 || storage > 2 || !(rho0 > 0.0)) {
        set_error("lbm_sums_noalloc: unknown storage or rho0 <= 0");
        return LBM_EINVAL;
    }
    int nb = reduce_blocks(nx, ny);
    if (nb > kMaxBlocks) {  // defensive: reduce_blocks caps at kReduceBlocksMax
        set_error("lbm_sums_noalloc: grid needs more reduction blocks than the scratch holds");
        return LBM_EINVAL;
    }
    double *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != LBM_OK) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double *partials = scratch;
    double *result = scratch + 3 * kMaxBlocks;
    cudaError_t e = launch_sums(storage, f, nx, ny, plane_stride, partials, result, st);
    double host[3];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host, result, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error(std::string("lbm_sums_noalloc: ") + cudaGetErrorString(e));
        return LBM_ECUDA;
    }
    out3[0] = (double)nx * (double)ny * rho0 + host[0];
    out3[1] = host[1];
    out3[2] = host[2];
    for (int k = 0; k < 3; ++k)
        if (!isfinite(out3[k])) {
            set_error("lbm_sums_noalloc: non-finite total");
            return LBM_ENONFINITE;
        }
    return LBM_OK;
}
