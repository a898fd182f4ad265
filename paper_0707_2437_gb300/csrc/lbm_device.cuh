// Device code of the fused variable-speed-of-sound D2Q9 step (sm_103a).
//
// One time step of Section 3, Eq. 5 (nbm) of Buick & Cosgrove:
//   f_i(x + e_i, t + 1) = f_i - (f_i - fbar_i)/tau + 3 w_i alpha grad(rho).e_i
// with fbar of Section 2, Eq. 2, rho and u of Eq. 3, alpha = 1/3 - c2
// (Eq. 8) and grad(rho) by central differences (Section 4).
//
// Layout.  Buffer = 9 planes (i = 0..8), plane stride P elements, each plane
// row-major [ny][nx].  A buffer holds the post-collision values f*_i(x, t-1)
// at their source site x (pull scheme): the pre-collision value at site x and
// time t is plane i at x - e_i.  One step reads buffer A and writes buffer B.
//
// Stored quantity.  h_i = (f_i - w_i rho0) / w_i.  In these variables the
// moments are  drho = rho - rho0 = sum_i w_i h_i,  j = rho u = sum_i w_i h_i e_i
// (the rest equilibrium carries no mass deviation and no momentum), and the
// update of Eq. 5 divided by w_i is
//   h*_i = (1 - 1/tau) h_i + (1/tau) Q_i + 3 alpha e_i.grad(rho)
//   Q_i  = drho + 3 e_i.j + 9/2 (e_i.j)(e_i.u) - 3/2 j.u        (= (fbar_i - w_i rho0)/w_i)
// Every stored value is then of the size of the density deviation, which keeps
// FP32 and 16-bit storage accurate for small waves.
//
// All arithmetic is FP32 with explicit round-to-nearest intrinsics, so the
// compiler cannot contract or reorder it differently in different
// instantiations: every tile configuration, the single-grid kernel and the
// batched kernel give bitwise identical results.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace vss {

enum Storage : int { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };

constexpr unsigned FULL = 0xffffffffu;

// Link vectors of Section 2: e_1..4 along the axes, e_5..8 the diagonals.
__host__ __device__ constexpr int EXi(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int EYi(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}

// Weights of Section 2 rounded to FP32.
#define VSS_W0 (4.0f / 9.0f)
#define VSS_W1 (1.0f / 9.0f)
#define VSS_W5 (1.0f / 36.0f)

// Per-grid constants of the collision.
struct Coef {
    float om;    // 1/tau
    float om1;   // 1 - 1/tau
    float w3;    // 3/tau
    float w45;   // 4.5/tau
    float a15;   // 1.5 alpha  (3 alpha times the 1/2 of the central difference)
    float rho0;  // reference density of the stored deviations
};

// ---------------------------------------------------------------------------
// Storage: a lane's V adjacent elements of one plane row are kept as NW 32-bit
// words: FP32 one element per word; 16-bit two elements per word (element 2k
// in the low half), or one element in the low half when V == 1.

template <int S>
struct StoreT;
template <>
struct StoreT<ST_F32> {
    using T = float;
};
template <>
struct StoreT<ST_F16> {
    using T = __half;
};
template <>
struct StoreT<ST_BF16> {
    using T = __nv_bfloat16;
};

template <int S, int V>
struct Pack {
    static constexpr int NW = (S == ST_F32) ? V : (V == 1 ? 1 : V / 2);
    static constexpr int BYTES = V * (S == ST_F32 ? 4 : 2);
};

template <int BYTES>
struct RawVec;
template <>
struct RawVec<2> {
    using T = unsigned short;
};
template <>
struct RawVec<4> {
    using T = unsigned int;
};
template <>
struct RawVec<8> {
    using T = uint2;
};
template <>
struct RawVec<16> {
    using T = uint4;
};

// Load policies.  LD_NC: the read-only (non-coherent) path, for kernels whose
// input buffer is not written while they run.  LD_CG: cached in L2 only, for
// the persistent batch kernel, whose buffers are rewritten by other blocks
// between its time steps.
enum LoadPolicy : int { LD_NC = 0, LD_CG = 1 };

template <int LD, typename R>
__device__ __forceinline__ R ld_policy(const R *p) {
    if constexpr (LD == LD_NC)
        return __ldg(p);
    else
        return __ldcg(p);
}

// Loads V elements into packed words.
template <int S, int V, int LD>
__device__ __forceinline__ void load_words(const void *p, uint32_t (&w)[Pack<S, V>::NW]) {
    constexpr int B = Pack<S, V>::BYTES;
    using R = typename RawVec<B>::T;
    R r = ld_policy<LD>(reinterpret_cast<const R *>(p));
    if constexpr (B == 2) {
        w[0] = (uint32_t)r;
    } else if constexpr (B == 4) {
        w[0] = r;
    } else if constexpr (B == 8) {
        w[0] = r.x;
        w[1] = r.y;
    } else {
        w[0] = r.x;
        w[1] = r.y;
        w[2] = r.z;
        w[3] = r.w;
    }
}

template <int S, int V>
__device__ __forceinline__ void store_words(void *p, const uint32_t (&w)[Pack<S, V>::NW]) {
    constexpr int B = Pack<S, V>::BYTES;
    using R = typename RawVec<B>::T;
    R r;
    if constexpr (B == 2) {
        r = (unsigned short)w[0];
    } else if constexpr (B == 4) {
        r = w[0];
    } else if constexpr (B == 8) {
        r = make_uint2(w[0], w[1]);
    } else {
        r = make_uint4(w[0], w[1], w[2], w[3]);
    }
    *reinterpret_cast<R *>(p) = r;
}

// One element (for the halo lanes): loaded into the low bits of a word.
template <int S, int LD>
__device__ __forceinline__ uint32_t load_elem(const void *p) {
    if constexpr (S == ST_F32)
        return ld_policy<LD>(reinterpret_cast<const unsigned int *>(p));
    else
        return (uint32_t)ld_policy<LD>(reinterpret_cast<const unsigned short *>(p));
}

// Element (low half / full word) to float.
template <int S>
__device__ __forceinline__ float elem_to_f(uint32_t e) {
    if constexpr (S == ST_F32)
        return __uint_as_float(e);
    else if constexpr (S == ST_F16)
        return __half2float(__ushort_as_half((unsigned short)(e & 0xffffu)));
    else
        return __uint_as_float(e << 16);
}

// Element v of a packed row as float.
template <int S, int V>
__device__ __forceinline__ float get_elem(const uint32_t (&w)[Pack<S, V>::NW], int v) {
    if constexpr (S == ST_F32) {
        return __uint_as_float(w[v]);
    } else if constexpr (V == 1) {
        return elem_to_f<S>(w[0]);
    } else {
        uint32_t x = w[v >> 1];
        return elem_to_f<S>((v & 1) ? (x >> 16) : x);
    }
}

// Float pair to a packed word (round to nearest even).
template <int S>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    if constexpr (S == ST_F16) {
        __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}
template <int S>
__device__ __forceinline__ uint32_t pack1(float v) {
    if constexpr (S == ST_F32) {
        return __float_as_uint(v);
    } else if constexpr (S == ST_F16) {
        return (uint32_t)__half_as_ushort(__float2half_rn(v));
    } else {
        return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
}

// Shifts of a lane's packed row by one element.  shift_from_left: element v
// takes element v-1 and element 0 takes `in`, the word that holds the left
// neighbour's last element (in its high half for 16-bit with V >= 2).
// shift_from_right: element v takes element v+1 and element V-1 takes `in`,
// the word that holds the right neighbour's first element (low half).
template <int S, int V>
__device__ __forceinline__ void shift_from_left(uint32_t (&w)[Pack<S, V>::NW], uint32_t in) {
    constexpr int NW = Pack<S, V>::NW;
    if constexpr (S == ST_F32 || V == 1) {
#pragma unroll
        for (int k = NW - 1; k > 0; --k) w[k] = w[k - 1];
        w[0] = in;
    } else {
#pragma unroll
        for (int k = NW - 1; k > 0; --k) w[k] = __byte_perm(w[k - 1], w[k], 0x5432);
        w[0] = __byte_perm(in, w[0], 0x5432);
    }
}
template <int S, int V>
__device__ __forceinline__ void shift_from_right(uint32_t (&w)[Pack<S, V>::NW], uint32_t in) {
    constexpr int NW = Pack<S, V>::NW;
    if constexpr (S == ST_F32 || V == 1) {
#pragma unroll
        for (int k = 0; k < NW - 1; ++k) w[k] = w[k + 1];
        w[NW - 1] = in;
    } else {
#pragma unroll
        for (int k = 0; k < NW - 1; ++k) w[k] = __byte_perm(w[k], w[k + 1], 0x5432);
        w[NW - 1] = __byte_perm(w[NW - 1], in, 0x5432);
    }
}

// ---------------------------------------------------------------------------
// Site arithmetic.

// drho = sum_i w_i h_i in one fixed order (Section 2, Eq. 3).  Used for the
// lane's own sites and for the halo sites, so that both give the same bits.
__device__ __forceinline__ float delta_rho(float h0, float h1, float h2, float h3, float h4,
                                           float h5, float h6, float h7, float h8) {
    float sa = __fadd_rn(__fadd_rn(h1, h2), __fadd_rn(h3, h4));
    float sd = __fadd_rn(__fadd_rn(h5, h6), __fadd_rn(h7, h8));
    return __fmaf_rn(VSS_W0, h0, __fmaf_rn(VSS_W1, sa, __fmul_rn(VSS_W5, sd)));
}

// Site quantities the nine outputs share.
struct SiteQ {
    float jx, jy, ux, uy;  // momentum rho u and velocity u (Eq. 3)
    float wB;              // (1/tau) (drho - 3/2 j.u)
    float Ax, Ay;          // 3 j/tau + 3 alpha grad(rho)
};

// dr: drho at the site; dxm/dxp, dym/dyp: drho at x -/+ 1 and y -/+ 1.
__device__ __forceinline__ SiteQ site_quantities(float h1, float h2, float h3, float h4, float h5,
                                                 float h6, float h7, float h8, float dr, float dxm,
                                                 float dxp, float dym, float dyp, const Coef &c) {
    SiteQ q;
    float a = __fsub_rn(h5, h7);  // e_5 = (1, 1), e_7 = -e_5
    float b = __fsub_rn(h6, h8);  // e_6 = (-1, 1), e_8 = -e_6
    q.jx = __fmaf_rn(VSS_W1, __fsub_rn(h1, h3), __fmul_rn(VSS_W5, __fsub_rn(a, b)));
    q.jy = __fmaf_rn(VSS_W1, __fsub_rn(h2, h4), __fmul_rn(VSS_W5, __fadd_rn(a, b)));
    float inv = __frcp_rn(__fadd_rn(c.rho0, dr));
    q.ux = __fmul_rn(q.jx, inv);
    q.uy = __fmul_rn(q.jy, inv);
    float ju = __fmaf_rn(q.jx, q.ux, __fmul_rn(q.jy, q.uy));
    q.wB = __fmul_rn(c.om, __fmaf_rn(-1.5f, ju, dr));
    // Central differences of Section 4: grad = (d(+1) - d(-1))/2; the 1/2 is in a15.
    q.Ax = __fmaf_rn(c.w3, q.jx, __fmul_rn(c.a15, __fsub_rn(dxp, dxm)));
    q.Ay = __fmaf_rn(c.w3, q.jy, __fmul_rn(c.a15, __fsub_rn(dyp, dym)));
    return q;
}

// Outputs of the pair (i, opposite of i) given e_i.j, e_i.u, e_i.A.
__device__ __forceinline__ void pair_out(float hi, float hopp, float ej, float eu, float eA,
                                         float wB, const Coef &c, float &oi, float &oopp) {
    float s = __fmaf_rn(c.w45, __fmul_rn(ej, eu), wB);
    oi = __fadd_rn(__fmaf_rn(c.om1, hi, s), eA);
    oopp = __fsub_rn(__fmaf_rn(c.om1, hopp, s), eA);
}

// ---------------------------------------------------------------------------
// The strip walk: one warp advances the sites x0 .. x0+32V-1 (clipped to nx)
// of rows y0 .. y1-1 by one step.  Each lane owns V adjacent sites.  The warp
// walks down the rows; for every row it pulls the nine distributions (Eq. 5,
// left-hand side) of its sites, forms drho, and collides the row above using
// drho of the rows above and below it (the y part of the central gradient,
// carried in registers) and of the lanes to its left and right (the x part,
// by warp shuffles).  Two halo columns (x0-1 and the column after the strip)
// are pulled by eight-plus-eight helper lanes so that the strip edges see the
// same drho their owners compute.  nx must be a multiple of V.
//
// Helper lanes (one load each per row):
//   lanes  0..8  : pulled f_i at (x0-1, row), i = lane
//   lanes  9..11 : f_i at column x0-1 for the three directions with e_x = +1
//                  (the left neighbour value lane 0 needs for its pull)
//   lanes 16..24 : pulled f_i at the column after the strip, i = lane - 16
//   lanes 25..27 : f_i at that column for the directions with e_x = -1
template <int S, int V, int LD = LD_NC>
struct Walker {
    static constexpr int NW = Pack<S, V>::NW;
    using T = typename StoreT<S>::T;

    const T *__restrict__ fin;
    T *__restrict__ fout;
    int nx, ny;
    size_t P;
    int x0, nact, lane, xs;
    bool act;
    // helper lane
    int gdir, gcol, gey;

    __device__ __forceinline__ Walker(const void *fin_, void *fout_, int nx_, int ny_, size_t P_,
                                      int x0_)
        : fin(reinterpret_cast<const T *>(fin_)),
          fout(reinterpret_cast<T *>(fout_)),
          nx(nx_),
          ny(ny_),
          P(P_),
          x0(x0_) {
        lane = threadIdx.x & 31;
        int wa = min(32 * V, nx - x0);
        nact = wa / V;
        act = lane < nact;
        xs = x0 + lane * V;
        int xl = (x0 == 0) ? nx - 1 : x0 - 1;
        int xr = (x0 + wa == nx) ? 0 : x0 + wa;
        gdir = -1;
        gcol = 0;
        if (lane < 9) {
            gdir = lane;
            gcol = xl - EXi(lane);
        } else if (lane < 12) {
            gdir = (lane == 9) ? 1 : (lane == 10 ? 5 : 8);
            gcol = xl;
        } else if (lane >= 16 && lane < 25) {
            gdir = lane - 16;
            gcol = xr - EXi(gdir);
        } else if (lane >= 25 && lane < 28) {
            gdir = (lane == 25) ? 3 : (lane == 26 ? 6 : 7);
            gcol = xr;
        }
        if (gcol < 0) gcol += nx;
        if (gcol >= nx) gcol -= nx;
        gey = gdir >= 0 ? EYi(gdir) : 0;
    }

    // Pulls row q (source rows qm = q-1, q0 = q, qp = q+1, already wrapped):
    // the lane's nine packed rows `w` (pre-collision f at its sites), drho of
    // its sites, and drho of the left / right halo sites (valid in every lane).
    __device__ __forceinline__ void pull_row(int qm, int q0, int qp, uint32_t (&w)[9][NW],
                                             float (&d)[V], float &dl, float &dr) const {
        // Source row of direction i is q - e_y(i).
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sr = (EYi(i) > 0) ? qm : ((EYi(i) < 0) ? qp : q0);
            if (act) {
                load_words<S, V, LD>(fin + (size_t)i * P + (size_t)sr * nx + xs, w[i]);
            } else {
#pragma unroll
                for (int k = 0; k < NW; ++k) w[i][k] = 0u;
            }
        }
        uint32_t g = 0u;
        if (gdir >= 0) {
            const int sr = (gey > 0) ? qm : ((gey < 0) ? qp : q0);
            g = load_elem<S, LD>(fin + (size_t)gdir * P + (size_t)sr * nx + gcol);
        }
        // e_x = +1 directions take the left neighbour's last element.
        {
            uint32_t e1 = __shfl_sync(FULL, g, 9);
            uint32_t e5 = __shfl_sync(FULL, g, 10);
            uint32_t e8 = __shfl_sync(FULL, g, 11);
            constexpr bool HI = (S != ST_F32 && V > 1);  // incoming element in the high half
            uint32_t p1 = __shfl_up_sync(FULL, w[1][NW - 1], 1);
            uint32_t p5 = __shfl_up_sync(FULL, w[5][NW - 1], 1);
            uint32_t p8 = __shfl_up_sync(FULL, w[8][NW - 1], 1);
            if (lane == 0) {
                p1 = HI ? (e1 << 16) : e1;
                p5 = HI ? (e5 << 16) : e5;
                p8 = HI ? (e8 << 16) : e8;
            }
            shift_from_left<S, V>(w[1], p1);
            shift_from_left<S, V>(w[5], p5);
            shift_from_left<S, V>(w[8], p8);
        }
        // e_x = -1 directions take the right neighbour's first element.
        {
            uint32_t e3 = __shfl_sync(FULL, g, 25);
            uint32_t e6 = __shfl_sync(FULL, g, 26);
            uint32_t e7 = __shfl_sync(FULL, g, 27);
            uint32_t n3 = __shfl_down_sync(FULL, w[3][0], 1);
            uint32_t n6 = __shfl_down_sync(FULL, w[6][0], 1);
            uint32_t n7 = __shfl_down_sync(FULL, w[7][0], 1);
            if (lane == nact - 1) {
                n3 = e3;
                n6 = e6;
                n7 = e7;
            }
            shift_from_right<S, V>(w[3], n3);
            shift_from_right<S, V>(w[6], n6);
            shift_from_right<S, V>(w[7], n7);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            d[v] = delta_rho(get_elem<S, V>(w[0], v), get_elem<S, V>(w[1], v),
                             get_elem<S, V>(w[2], v), get_elem<S, V>(w[3], v),
                             get_elem<S, V>(w[4], v), get_elem<S, V>(w[5], v),
                             get_elem<S, V>(w[6], v), get_elem<S, V>(w[7], v),
                             get_elem<S, V>(w[8], v));
        }
        // Halo drho: lanes 0..8 hold the left halo's nine values, 16..24 the
        // right halo's; gather them in direction order and sum as above.
        {
            const int base = lane & 16;
            float hh[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) hh[i] = elem_to_f<S>(__shfl_sync(FULL, g, base + i));
            float dh = delta_rho(hh[0], hh[1], hh[2], hh[3], hh[4], hh[5], hh[6], hh[7], hh[8]);
            dl = __shfl_sync(FULL, dh, 0);
            dr = __shfl_sync(FULL, dh, 16);
        }
    }

    // Collides row r (packed pulled values w, drho d of the row, du / dd of the
    // rows above / below, dl / dr of the halo sites) and stores it.
    __device__ __forceinline__ void collide_store(int r, const uint32_t (&w)[9][NW],
                                                  const float (&d)[V], const float (&dym)[V],
                                                  const float (&dyp)[V], float dl, float dr,
                                                  const Coef &c) const {
        // x neighbours of drho: inside the lane, then the adjacent lanes, then
        // the halo sites at the strip edges.
        float lft = __shfl_up_sync(FULL, d[V - 1], 1);
        float rgt = __shfl_down_sync(FULL, d[0], 1);
        if (lane == 0) lft = dl;
        if (lane == nact - 1) rgt = dr;

        SiteQ q[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            float dxm = (v == 0) ? lft : d[v - 1];
            float dxp = (v == V - 1) ? rgt : d[v + 1];
            q[v] = site_quantities(get_elem<S, V>(w[1], v), get_elem<S, V>(w[2], v),
                                   get_elem<S, V>(w[3], v), get_elem<S, V>(w[4], v),
                                   get_elem<S, V>(w[5], v), get_elem<S, V>(w[6], v),
                                   get_elem<S, V>(w[7], v), get_elem<S, V>(w[8], v), d[v], dxm,
                                   dxp, dym[v], dyp[v], c);
        }
        const size_t row = (size_t)r * nx + xs;
        float o0[V], oa[V], ob[V];
        // Direction 0 (rest).
#pragma unroll
        for (int v = 0; v < V; ++v) o0[v] = __fmaf_rn(c.om1, get_elem<S, V>(w[0], v), q[v].wB);
        store_dir(0, row, o0);
        // (1, 3): e = (1, 0).
#pragma unroll
        for (int v = 0; v < V; ++v)
            pair_out(get_elem<S, V>(w[1], v), get_elem<S, V>(w[3], v), q[v].jx, q[v].ux, q[v].Ax,
                     q[v].wB, c, oa[v], ob[v]);
        store_dir(1, row, oa);
        store_dir(3, row, ob);
        // (2, 4): e = (0, 1).
#pragma unroll
        for (int v = 0; v < V; ++v)
            pair_out(get_elem<S, V>(w[2], v), get_elem<S, V>(w[4], v), q[v].jy, q[v].uy, q[v].Ay,
                     q[v].wB, c, oa[v], ob[v]);
        store_dir(2, row, oa);
        store_dir(4, row, ob);
        // (5, 7): e = (1, 1).
#pragma unroll
        for (int v = 0; v < V; ++v)
            pair_out(get_elem<S, V>(w[5], v), get_elem<S, V>(w[7], v),
                     __fadd_rn(q[v].jx, q[v].jy), __fadd_rn(q[v].ux, q[v].uy),
                     __fadd_rn(q[v].Ax, q[v].Ay), q[v].wB, c, oa[v], ob[v]);
        store_dir(5, row, oa);
        store_dir(7, row, ob);
        // (6, 8): e = (-1, 1).
#pragma unroll
        for (int v = 0; v < V; ++v)
            pair_out(get_elem<S, V>(w[6], v), get_elem<S, V>(w[8], v),
                     __fsub_rn(q[v].jy, q[v].jx), __fsub_rn(q[v].uy, q[v].ux),
                     __fsub_rn(q[v].Ay, q[v].Ax), q[v].wB, c, oa[v], ob[v]);
        store_dir(6, row, oa);
        store_dir(8, row, ob);
    }

    __device__ __forceinline__ void store_dir(int i, size_t row, const float (&o)[V]) const {
        if (!act) return;
        uint32_t pw[NW];
        if constexpr (S == ST_F32 || V == 1) {
#pragma unroll
            for (int v = 0; v < V; ++v) pw[v] = pack1<S>(o[v]);
        } else {
#pragma unroll
            for (int k = 0; k < NW; ++k) pw[k] = pack2<S>(o[2 * k], o[2 * k + 1]);
        }
        store_words<S, V>(fout + (size_t)i * P + row, pw);
    }

    // Advances rows y0 .. y1-1 (0 <= y0 < y1 <= ny) by one step.
    __device__ __forceinline__ void run(int y0, int y1, const Coef &c) const {
        // Pulled-row cursor: q and its source rows q-1, q+1, all wrapped.
        int q0 = (y0 == 0) ? ny - 1 : y0 - 1;
        int qm = (q0 == 0) ? ny - 1 : q0 - 1;
        int qp = (q0 + 1 == ny) ? 0 : q0 + 1;

        uint32_t wc[9][NW], wn[9][NW];
        float dprev[V], dcur[V], dnext[V];
        float dlc, drc, dln, drn;

        pull_row(qm, q0, qp, wn, dprev, dln, drn);  // row y0 - 1: drho only
        qm = q0;
        q0 = qp;
        qp = (qp + 1 == ny) ? 0 : qp + 1;
        pull_row(qm, q0, qp, wc, dcur, dlc, drc);  // row y0
        for (int r = y0; r < y1; ++r) {
            qm = q0;
            q0 = qp;
            qp = (qp + 1 == ny) ? 0 : qp + 1;
            pull_row(qm, q0, qp, wn, dnext, dln, drn);  // row r + 1
            collide_store(r, wc, dcur, dprev, dnext, dlc, drc, c);
#pragma unroll
            for (int i = 0; i < 9; ++i)
#pragma unroll
                for (int k = 0; k < NW; ++k) wc[i][k] = wn[i][k];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                dprev[v] = dcur[v];
                dcur[v] = dnext[v];
            }
            dlc = dln;
            drc = drn;
        }
    }
};

}  // namespace vss
