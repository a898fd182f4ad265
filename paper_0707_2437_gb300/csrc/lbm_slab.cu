// Slab decomposition of one grid in y (several GPUs, one slab each).
//
// Rank r of N owns the global rows [r*ny_local, (r+1)*ny_local).  Its
// handle's buffers hold ny_local + 4 rows: ghost rows 0 and 1 (the two rows
// below its own, owned by rank r-1), its own rows 2 .. ny_local+1, and ghost
// rows ny_local+2 and ny_local+3 (the two rows above, owned by rank r+1),
// with ranks wrapping around (the grid stays periodic in y).  A step of
// Eq. 5 at a row reads the stored values of the rows up to two away (the
// pull reaches one row, the central gradient of the pulled density one
// more), so two ghost rows suffice.  A step computes the own rows only (the
// batch work-list covers them alone, and no pull wraps in y), and between
// steps each rank sends its two lowest own rows to rank r-1 and its two
// highest to rank r+1, all nine planes: 2 * 9 * nx elements a side.  The
// exchange itself is the caller's (for example NCCL send/recv of the packed
// rows); the library packs and unpacks them on the handle's stream.
#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace vss;

static constexpr int kGhost = 2;

extern "C" int lbm_slab_create(int nx, int ny_local, double tau, double c2, int storage,
                               void *cuda_stream, lbm_t *out) {
    if (!out) {
        set_error("lbm_slab_create: out is NULL");
        return LBM_EINVAL;
    }
    *out = nullptr;
    if (ny_local < kGhost || ny_local > 0x7fffffff - 2 * kGhost) {
        set_error("lbm_slab_create: need ny_local >= 2 (the rows a neighbour reads)");
        return LBM_EINVAL;
    }
    lbm_t h = nullptr;
    int rc = lbm_create(nx, ny_local + 2 * kGhost, tau, c2, storage, cuda_stream, &h);
    if (rc < 0) return rc;
    h->slab = kGhost;
    *out = h;
    return rc;
}

extern "C" size_t lbm_slab_halo_bytes(lbm_t h) {
    if (!h || !h->slab) return 0;
    return (size_t)9 * kGhost * (size_t)h->nx * (size_t)elem_bytes(h->storage);
}

// Rows [row, row + 2) of all nine planes of the current state, to or from a
// packed [9][2][nx] device buffer.
static int slab_copy(lbm_t h, void *packed, int side, bool pack, const char *what) {
    if (!h || !packed || (side != 0 && side != 1)) {
        set_error(std::string(what) + ": bad argument");
        return LBM_EINVAL;
    }
    if (!h->slab) {
        set_error(std::string(what) + ": not a slab handle");
        return LBM_EINVAL;
    }
    const size_t eb = (size_t)elem_bytes(h->storage);
    const size_t width = (size_t)kGhost * h->nx * eb;  // two rows
    int row;
    if (pack)
        row = side == 0 ? kGhost : h->ny - 2 * kGhost;  // own rows next to that side
    else
        row = side == 0 ? 0 : h->ny - kGhost;           // that side's ghost rows
    unsigned char *state = static_cast<unsigned char *>(h->buf[h->cur]) + (size_t)row * h->nx * eb;
    cudaError_t e;
    if (pack)
        e = cudaMemcpy2DAsync(packed, width, state, h->P * eb, width, 9, cudaMemcpyDeviceToDevice,
                              h->stream);
    else
        e = cudaMemcpy2DAsync(state, h->P * eb, packed, width, width, 9, cudaMemcpyDeviceToDevice,
                              h->stream);
    if (e != cudaSuccess) {
        set_error(std::string(what) + ": " + cudaGetErrorString(e));
        return LBM_ECUDA;
    }
    return LBM_OK;
}

extern "C" int lbm_slab_pack(lbm_t h, void *dst, int side) {
    return slab_copy(h, dst, side, true, "lbm_slab_pack");
}

extern "C" int lbm_slab_unpack(lbm_t h, const void *src, int side) {
    return slab_copy(h, const_cast<void *>(src), side, false, "lbm_slab_unpack");
}
