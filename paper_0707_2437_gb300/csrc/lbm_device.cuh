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

#ifdef VSS_BOUNDS_CHECK
// Debug builds only: every global access of the walk checks its element
// index against the buffer; a violation is counted (and its first index kept)
// in this translation unit's record and the access is skipped.
static __device__ unsigned long long vss_oob_record[2];
__device__ __forceinline__ bool vss_in_bounds(size_t idx, size_t n, size_t lim) {
    if (idx + n <= lim) return true;
    if (atomicAdd(&vss_oob_record[0], 1ULL) == 0ULL) vss_oob_record[1] = idx;
    return false;
}
#define VSS_IN_BOUNDS(idx, n, lim) vss_in_bounds((idx), (n), (lim))
#else
#define VSS_IN_BOUNDS(idx, n, lim) true
#endif

constexpr unsigned FULL = 0xffffffffu;

// Link vectors of Section 2: e_1..4 along the axes, e_5..8 the diagonals.
__host__ __device__ constexpr int EXi(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int EYi(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}

// Weights of Section 2 in FP32, chosen so that the collision conserves the
// density and momentum deviations exactly in its linear part: W1 = fl(1/9),
// W5 = 1/36 on the 2^-27 grid, and W0 = 1 - 4 W1 - 4 W5 (which is 4 W1), so
// that W0 + 4 W1 + 4 W5 = 1 exactly; each is within 1e-7 of the printed
// weight.  (Rounded one by one they sum to 1 + 7.5e-9; together with
// 1 - 1/tau rounded apart from 1/tau, every step then scaled the density and
// momentum deviations by 1 + O(1e-7), 0.3 % over 40,000 steps.)
#define VSS_W0 0x1.c71c72p-2f
#define VSS_W1 0x1.c71c72p-4f
#define VSS_W5 0x1.c71c7p-6f
// T = 2 (W1 + 2 W5) = sum_i W_i e_ix^2 (1/3 - 5e-9), exact in double: the
// momentum a collision adds is T times the antisymmetric part it puts on
// each link pair.
#define VSS_T_D 0x1.555555p-2
// 1 / (2 T): 1.5 alpha scaled so that the force adds momentum alpha grad(rho)
// with these weights (the 1/2 of the central difference included).
#define VSS_A15_SCALE_D 0x1.8000006000002p+0

// The per-site force constant alpha / (2 T) in FP32 from alpha in FP64, the
// same rounding for a grid's uniform alpha (host) and a c2 field (device), so
// that a uniform field reproduces the uniform run bitwise.
__host__ __device__ inline float a15_of_alpha(double alpha) {
    return (float)(alpha * VSS_A15_SCALE_D);
}

// Per-grid constants of the collision.
struct Coef {
    float om;    // 1/tau
    float om1;   // 1 - 1/tau; om + om1 == 1 exactly in FP32
    float w3;    // 3/tau as (1/tau)/T, split into a rounded value ...
    float w3lo;  // ... and its remainder, so that T (w3 + w3lo) = 1/tau to ~2^-48
    float w45;   // 4.5/tau
    float a15;   // alpha / (2 T), about 1.5 alpha (3 alpha times the 1/2 of the
                 // central difference)
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

// Element v of a packed row set from a float (round to nearest even for the
// 16-bit kinds; each element is rounded on its own).
template <int S>
__device__ __forceinline__ uint32_t pack1(float v);
template <int S, int V>
__device__ __forceinline__ void set_elem(uint32_t (&w)[Pack<S, V>::NW], int v, float x) {
    if constexpr (S == ST_F32) {
        w[v] = __float_as_uint(x);
    } else if constexpr (V == 1) {
        w[0] = pack1<S>(x);
    } else {
        const uint32_t b = pack1<S>(x);
        w[v >> 1] = (v & 1) ? __byte_perm(w[v >> 1], b, 0x5410) : __byte_perm(w[v >> 1], b, 0x3254);
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
    // The paired conversion (same rounding) with the value in the low half.
    if constexpr (S == ST_F32)
        return __float_as_uint(v);
    else
        return pack2<S>(v, 0.0f) & 0xffffu;
}

// ---------------------------------------------------------------------------
// Stochastic rounding of the 16-bit stores (optional).  With round to nearest
// a stored value that changes by less than half a unit in the last place per
// step never changes at all, which freezes slow processes such as the viscous
// decay of long shear waves.  Stochastic rounding rounds up with probability
// equal to the discarded fraction (as many random bits as dropped bits), so the expected
// stored value equals the FP32 result.  The random bits are a counter-based
// hash of (site, step): deterministic, and independent of the tile
// configuration and of batching, so results stay bitwise reproducible.

// 32-bit integer mixing function (xor-shift / multiply, the "lowbias32"
// constants found by Wellons' hash prospector).
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Random bits for stochastic rounding, from a counter-based hash of (pair of
// sites, direction, step): one 32-bit word per direction for the sites 2p and
// 2p+1 of the grid's row-major order (p = site >> 1); its low half rounds site
// 2p and its high half site 2p+1.  The word depends on nothing else, so runs
// are deterministic and independent of tile shape, sites per lane and
// batching (with 2, 4 or 8 sites per lane nx is even, so the two sites of a
// packed word are always such a pair; a 1-site lane takes its half).  The
// pair hash is the full mix.  A direction's word is that hash times an odd
// constant of its own (a bijection of the 32-bit words, different for every
// direction), with the high half folded into the low one so that the low
// bits, which FP16 uses, depend on every bit of the hash: three instructions
// per word.
__device__ __forceinline__ uint32_t sr_step_key(uint32_t step) {
    return mix32(step * 0x9e3779b9u + 0x632be5abu);
}
__device__ __forceinline__ uint32_t sr_pair_base(uint32_t site, uint32_t key) {
    return mix32((site >> 1) ^ key);
}
__device__ __forceinline__ uint32_t sr_word(uint32_t base, int i) {
    const uint32_t x = base * (0x9e3779b9u + 2u * (uint32_t)i * 0x6a09e667u);
    return x ^ (x >> 16);
}

// FP32 -> 16-bit with round up probability equal to the discarded fraction,
// on the stochastic-rounding conversions of sm_100-class GPUs (PTX cvt with
// .rs rounding): the conversion adds the caller's random bits to the bits
// the 16-bit format drops and truncates (FP16 drops 13 bits and takes the low
// 13 random bits of its half of rbits, BF16 drops 16 and takes all 16; the
// low half of rbits rounds the low element).  With as many random bits as
// dropped bits the rounding is exactly unbiased.  One instruction converts a
// pair of elements.
template <int S>
__device__ __forceinline__ uint32_t sr_pack2(float lo, float hi, uint32_t rbits) {
    uint32_t out;
    if constexpr (S == ST_F16)
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(out) : "f"(hi), "f"(lo), "r"(rbits));
    else
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(out) : "f"(hi), "f"(lo), "r"(rbits));
    return out;
}

// One element (in the low half of the result), with the 16 random bits `r`.
template <int S>
__device__ __forceinline__ uint32_t sr_round(float x, uint32_t r) {
    return sr_pack2<S>(x, 0.0f, r & 0xffffu) & 0xffffu;
}

// Sites per packed word: the 16-bit kinds convert two sites at a time.
template <int S, int V>
struct SitesPerWord {
    static constexpr int value = (S == ST_F32 || V == 1) ? 1 : 2;
};

// Both elements of a packed 16-bit word as floats (element 2k in .x).
template <int S>
__device__ __forceinline__ float2 unpack2(uint32_t w) {
    if constexpr (S == ST_F16) {
        __half2 h = *reinterpret_cast<__half2 *>(&w);
        return __half22float2(h);
    } else {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
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

// 1/x by the hardware reciprocal (rcp.approx.ftz.f32: about 1 ulp, one
// instruction).  Only u = j/rho uses it; u is of the size of the wave's
// velocity, so the absolute error stays near 1e-7 |u|.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
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
                                                 float dxp, float dym, float dyp, const Coef &c,
                                                 float a15) {
    SiteQ q;
    float a = __fsub_rn(h5, h7);  // e_5 = (1, 1), e_7 = -e_5
    float b = __fsub_rn(h6, h8);  // e_6 = (-1, 1), e_8 = -e_6
    q.jx = __fmaf_rn(VSS_W1, __fsub_rn(h1, h3), __fmul_rn(VSS_W5, __fsub_rn(a, b)));
    q.jy = __fmaf_rn(VSS_W1, __fsub_rn(h2, h4), __fmul_rn(VSS_W5, __fadd_rn(a, b)));
    float inv = rcp_approx(__fadd_rn(c.rho0, dr));
    q.ux = __fmul_rn(q.jx, inv);
    q.uy = __fmul_rn(q.jy, inv);
    float ju = __fmaf_rn(q.jx, q.ux, __fmul_rn(q.jy, q.uy));
    q.wB = __fmul_rn(c.om, __fmaf_rn(-1.5f, ju, dr));
    // Central differences of Section 4: grad = (d(+1) - d(-1))/2; the 1/2 is in a15.
    q.Ax = __fmaf_rn(c.w3, q.jx, __fmaf_rn(c.w3lo, q.jx, __fmul_rn(a15, __fsub_rn(dxp, dxm))));
    q.Ay = __fmaf_rn(c.w3, q.jy, __fmaf_rn(c.w3lo, q.jy, __fmul_rn(a15, __fsub_rn(dyp, dym))));
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
// SEG = 32: the warp walks one strip of 32*V columns.  SEG = 16 (split walk):
// each half-warp walks its own segment of a strip at most 16*V columns wide,
// so that two narrow pieces of work fill one warp; every shuffle stays within
// the half, and each lane serves one halo role on each side.
// GR = 1: the forward difference the paper tried before the central one
// (Section 4): grad = rho(x+1) - rho(x) in x and y instead of half the central
// difference, for the instability it shows as c_e approaches 1.  Only the
// FP32 single-grid step kernel instantiates it.
template <int S, int V, int LD = LD_NC, int RND = 0, int VA = 0, int SEG = 32, int GR = 0>
struct Walker {
    static constexpr int NW = Pack<S, V>::NW;
    using T = typename StoreT<S>::T;
    static_assert(RND == 0 || S != ST_F32, "stochastic rounding applies to 16-bit storage");
    static_assert(SEG == 32 || SEG == 16, "a strip is walked by a warp or a half-warp");
    uint32_t rkey = 0;  // sr_step_key of the step number (stochastic rounding)
    __device__ __forceinline__ void set_step(uint32_t step) { rkey = sr_step_key(step); }
    // Spatially varying sound speed (VA = 1): 1.5 alpha per site, [ny][nx].
    const float *__restrict__ a15f = nullptr;

    const T *__restrict__ fin;
    T *__restrict__ fout;
    int nx, ny;
    size_t P;
    int x0, wa, nact, lane, sl, xs;
    bool act;
    // helper lane: direction, column offset from x0 (unwrapped), wrapped column
    int gdir, goff, gcol, gey;
    // split walk: the lane's right-side role (direction, wrapped column, e_y)
    int gdir2, gcol2, gey2;

    __device__ __forceinline__ Walker(const void *fin_, void *fout_, int nx_, int ny_, size_t P_,
                                      int x0_)
        : fin(reinterpret_cast<const T *>(fin_)),
          fout(reinterpret_cast<T *>(fout_)),
          nx(nx_),
          ny(ny_),
          P(P_),
          x0(x0_) {
        lane = threadIdx.x & 31;
        sl = lane & (SEG - 1);
        wa = min(SEG * V, nx - x0);
        nact = wa / V;
        act = sl < nact;
        xs = x0 + sl * V;
        if constexpr (SEG == 32) {
            helper_role(lane, gdir, goff, gcol, gey);
        } else {
            // Sub-lanes 0..11 of each half: the left roles of lanes 0..11 of a
            // whole-warp strip, and the right roles of lanes 16..27.
            int goff2;
            helper_role(sl, gdir, goff, gcol, gey);
            helper_role(sl + 16, gdir2, goff2, gcol2, gey2);
        }
        __syncwarp();
    }

    // Helper roles of lane `r` of a whole-warp strip, read from packed per-lane
    // tables without branches: direction (4 bits per lane) and kind (2 bits
    // per lane).
    //   kind 0: pulled f at the left halo site x0-1   (column x0-1-e_x)
    //   kind 1: f at column x0-1 (left edge value; lanes without a
    //           role also take kind 1, direction 0, and ignore it)
    //   kind 2: pulled f at the right halo site x0+wa (column x0+wa-e_x)
    //   kind 3: f at column x0+wa (right edge value)
    __device__ __forceinline__ void helper_role(int r, int &dir, int &off, int &col,
                                                int &ey) const {
        const unsigned long long dir_tab = (r < 16) ? 0x851876543210ULL : 0x763876543210ULL;
        dir = (int)((dir_tab >> (4 * (r & 15))) & 15ULL);
        const int kind = (int)((0x55feaaaa55540000ULL >> (2 * r)) & 3ULL);
        const int ex = (int)((0x20919u >> (2 * dir)) & 3u) - 1;  // e_x of dir
        const int base = (kind < 2) ? -1 : wa;
        off = base - (((kind & 1) == 0) ? ex : 0);
        col = ((x0 + off) % nx + nx) % nx;
        ey = (int)((0x2865u >> (2 * dir)) & 3u) - 1;  // e_y of dir
    }

    // Pulls row q (source rows qm = q-1, q0 = q, qp = q+1, already wrapped):
    // the lane's nine packed rows `w` (pre-collision f at its sites), drho of
    // its sites, and drho of the left / right halo sites (valid in every lane).
    __device__ __forceinline__ void pull_row(int qm, int q0, int qp, uint32_t (&w)[9][NW],
                                             float (&d)[V], float &dl, float &dr) const {
        uint32_t g;
        load_row(qm, q0, qp, w, g);
        finish_pull(w, g, d, dl, dr);
    }

    // The loads of a pull: the lane's nine aligned vectors and the helper value.
    __device__ __forceinline__ void load_row(int qm, int q0, int qp, uint32_t (&w)[9][NW],
                                             uint32_t &g) const {
        // Source row of direction i is q - e_y(i).
        // Lanes past the end of a partial strip load the strip's first
        // elements instead (unused), so that every lane issues the same loads.
        const int xl = act ? xs : x0;
        const size_t lim = 9 * P;
        (void)lim;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sr = (EYi(i) > 0) ? qm : ((EYi(i) < 0) ? qp : q0);
            const size_t idx = (size_t)i * P + (size_t)sr * nx + xl;
            if (VSS_IN_BOUNDS(idx, V, lim)) {
                load_words<S, V, LD>(fin + idx, w[i]);
            } else {
#pragma unroll
                for (int k = 0; k < NW; ++k) w[i][k] = 0u;
            }
        }
        const int gsr = (gey > 0) ? qm : ((gey < 0) ? qp : q0);
        const size_t gidx = (size_t)gdir * P + (size_t)gsr * nx + gcol;
        g = VSS_IN_BOUNDS(gidx, 1, lim) ? load_elem<S, LD>(fin + gidx) : 0u;
    }

    // The nine values of sites v0 .. v0+SP-1 as floats, and back (the 16-bit
    // kinds convert the two sites of a word together; rounding is per element).
    __device__ __forceinline__ static void unpack_sites(
        const uint32_t (&w)[9][NW], int v0, float (&h)[SitesPerWord<S, V>::value][9]) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if constexpr (SitesPerWord<S, V>::value == 2) {
                const float2 f = unpack2<S>(w[i][v0 >> 1]);
                h[0][i] = f.x;
                h[1][i] = f.y;
            } else {
                h[0][i] = get_elem<S, V>(w[i], v0);
            }
        }
    }
    __device__ __forceinline__ void pack_sites(
        uint32_t (&w)[9][NW], int v0, const float (&h)[SitesPerWord<S, V>::value][9],
        int r) const {
        constexpr int SP = SitesPerWord<S, V>::value;
        if constexpr (RND == 0) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                if constexpr (SP == 2)
                    w[i][v0 >> 1] = pack2<S>(h[0][i], h[1][i]);
                else
                    set_elem<S, V>(w[i], v0, h[0][i]);
            }
        } else {
            const uint32_t site = (uint32_t)r * (uint32_t)nx + (uint32_t)(xs + v0);
            const uint32_t base = sr_pair_base(site, rkey);
            if constexpr (SP == 2) {
                // site is even: the word's two sites are the pair (site, site + 1)
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    w[i][v0 >> 1] = sr_pack2<S>(h[0][i], h[1][i], sr_word(base, i));
            } else {
                const uint32_t sh = (site & 1u) * 16u;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const uint32_t b = sr_round<S>(h[0][i], sr_word(base, i) >> sh);
                    if constexpr (V == 1)
                        w[i][0] = b;
                    else
                        w[i][v0 >> 1] = (v0 & 1) ? __byte_perm(w[i][v0 >> 1], b, 0x5410)
                                                 : __byte_perm(w[i][v0 >> 1], b, 0x3254);
                }
            }
        }
    }

    // Shifts of the e_x = +-1 directions, drho of the lane's sites, and drho
    // of the two halo sites, from the raw rows `w` and the helper value `g`
    // (split walk: `g` of the lane's left role, `g2` of its right role).
    __device__ __forceinline__ void finish_pull(uint32_t (&w)[9][NW], uint32_t g, float (&d)[V],
                                                float &dl, float &dr, uint32_t g2 = 0u) const {
        // The right edge values: lanes 25..27 of the warp, or 9..11 of a half.
        const uint32_t gr = (SEG == 32) ? g : g2;
        constexpr int RE = (SEG == 32) ? 25 : 9;
        // e_x = +1 directions take the left neighbour's last element.
        {
            uint32_t e1 = __shfl_sync(FULL, g, 9, SEG);
            uint32_t e5 = __shfl_sync(FULL, g, 10, SEG);
            uint32_t e8 = __shfl_sync(FULL, g, 11, SEG);
            constexpr bool HI = (S != ST_F32 && V > 1);  // incoming element in the high half
            uint32_t p1 = __shfl_up_sync(FULL, w[1][NW - 1], 1, SEG);
            uint32_t p5 = __shfl_up_sync(FULL, w[5][NW - 1], 1, SEG);
            uint32_t p8 = __shfl_up_sync(FULL, w[8][NW - 1], 1, SEG);
            if (sl == 0) {
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
            uint32_t e3 = __shfl_sync(FULL, gr, RE, SEG);
            uint32_t e6 = __shfl_sync(FULL, gr, RE + 1, SEG);
            uint32_t e7 = __shfl_sync(FULL, gr, RE + 2, SEG);
            uint32_t n3 = __shfl_down_sync(FULL, w[3][0], 1, SEG);
            uint32_t n6 = __shfl_down_sync(FULL, w[6][0], 1, SEG);
            uint32_t n7 = __shfl_down_sync(FULL, w[7][0], 1, SEG);
            if (sl == nact - 1) {
                n3 = e3;
                n6 = e6;
                n7 = e7;
            }
            shift_from_right<S, V>(w[3], n3);
            shift_from_right<S, V>(w[6], n6);
            shift_from_right<S, V>(w[7], n7);
        }
        constexpr int SP = SitesPerWord<S, V>::value;
#pragma unroll
        for (int v0 = 0; v0 < V; v0 += SP) {
            float h[SP][9];
            unpack_sites(w, v0, h);
#pragma unroll
            for (int s = 0; s < SP; ++s)
                d[v0 + s] = delta_rho(h[s][0], h[s][1], h[s][2], h[s][3], h[s][4], h[s][5],
                                      h[s][6], h[s][7], h[s][8]);
        }
        // Halo drho: lanes 0..8 hold the left halo's nine values, 16..24 the
        // right halo's.  The sums of delta_rho are formed across lanes in the
        // same order: lanes 1, 3, 5, 7 add their right neighbour (h1+h2,
        // h3+h4, h5+h6, h7+h8), lanes 1 and 5 then add the pair two lanes on
        // ((h1+h2)+(h3+h4), (h5+h6)+(h7+h8)), and lane 0 (16) combines them
        // with h0 as delta_rho does.  Split walk: the same sums within each
        // half, once over the left roles and once over the right ones.
        if constexpr (SEG == 16) {
            dl = halo_drho16(g);
            dr = halo_drho16(g2);
        } else {
            const float v = elem_to_f<S>(g);
            const float t = __fadd_rn(v, __shfl_down_sync(FULL, v, 1));
            const float u = __fadd_rn(t, __shfl_down_sync(FULL, t, 2));
            const int base = lane & 16;
            const float sa = __shfl_sync(FULL, u, base + 1);
            const float sd = __shfl_sync(FULL, u, base + 5);
            const float dh = __fmaf_rn(VSS_W0, v, __fmaf_rn(VSS_W1, sa, __fmul_rn(VSS_W5, sd)));
            dl = __shfl_sync(FULL, dh, 0);
            dr = __shfl_sync(FULL, dh, 16);
        }
    }
    __device__ __forceinline__ static float halo_drho16(uint32_t g) {
        const float v = elem_to_f<S>(g);
        const float t = __fadd_rn(v, __shfl_down_sync(FULL, v, 1, 16));
        const float u = __fadd_rn(t, __shfl_down_sync(FULL, t, 2, 16));
        const float sa = __shfl_sync(FULL, u, 1, 16);
        const float sd = __shfl_sync(FULL, u, 5, 16);
        const float dh = __fmaf_rn(VSS_W0, v, __fmaf_rn(VSS_W1, sa, __fmul_rn(VSS_W5, sd)));
        return __shfl_sync(FULL, dh, 0, 16);
    }

    // Collides row r and stores it.  w: the row's packed pulled values (the
    // outputs are written back into it, site by site, and then stored); d:
    // drho of the row; dym / dyp: drho of rows r-1 / r+1; dl / dr: drho of
    // the halo sites left and right of the strip; keep = false computes the
    // row without storing it (the shorter half of a split walk); swap_y
    // exchanges dym and dyp (the halves of a split walk walk in opposite
    // directions: selecting the rows per lane keeps the warp on one path,
    // where a branch would run the halves one after the other).
    __device__ __forceinline__ void collide_store(int r, uint32_t (&w)[9][NW], const float (&d)[V],
                                                  const float (&dym)[V], const float (&dyp)[V],
                                                  float dl, float dr, const Coef &c,
                                                  bool keep = true, bool swap_y = false,
                                                  const uint4 *aslot = nullptr) const {
        // x neighbours of drho: inside the lane, then the adjacent lanes, then
        // the halo sites at the strip edges.
        float lft = __shfl_up_sync(FULL, d[V - 1], 1, SEG);
        float rgt = __shfl_down_sync(FULL, d[0], 1, SEG);
        if (sl == 0) lft = dl;
        if (sl == nact - 1) rgt = dr;
        // 1.5 alpha of the lane's sites: the grid's constant, or the field
        // (8-site walks: staged in shared memory by run_async, `aslot`, or
        // read as two 16-byte vectors).
        float a15v[V];
        if constexpr (VA && V == 8) {
            if (aslot) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint4 u = aslot[h * 32 + lane];
                    a15v[4 * h + 0] = __uint_as_float(u.x);
                    a15v[4 * h + 1] = __uint_as_float(u.y);
                    a15v[4 * h + 2] = __uint_as_float(u.z);
                    a15v[4 * h + 3] = __uint_as_float(u.w);
                }
            } else {
                const size_t aidx = (size_t)r * nx + (act ? xs : x0);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t aw[4];
                    if (VSS_IN_BOUNDS(aidx + 4 * h, 4, (size_t)nx * ny)) {
                        load_words<ST_F32, 4, LD>(a15f + aidx + 4 * h, aw);
                    } else {
#pragma unroll
                        for (int v = 0; v < 4; ++v) aw[v] = 0u;
                    }
#pragma unroll
                    for (int v = 0; v < 4; ++v) a15v[4 * h + v] = __uint_as_float(aw[v]);
                }
            }
        } else if constexpr (VA) {
            const size_t aidx = (size_t)r * nx + (act ? xs : x0);
            uint32_t aw[V];
            if (VSS_IN_BOUNDS(aidx, V, (size_t)nx * ny)) {
                load_words<ST_F32, V, LD>(a15f + aidx, aw);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) aw[v] = 0u;
            }
#pragma unroll
            for (int v = 0; v < V; ++v) a15v[v] = __uint_as_float(aw[v]);
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) a15v[v] = c.a15;
        }
        constexpr int SP = SitesPerWord<S, V>::value;
#pragma unroll
        for (int v0 = 0; v0 < V; v0 += SP) {
            float h[SP][9];
            unpack_sites(w, v0, h);
#pragma unroll
            for (int s = 0; s < SP; ++s) {
                const int v = v0 + s;
                // Forward difference: the site itself in place of the x-1 and
                // y-1 neighbours, and twice the factor that holds the central
                // difference's 1/2 (exact in FP32).
                const float dxm = GR ? d[v] : ((v == 0) ? lft : d[v - 1]);
                const float dxp = (v == V - 1) ? rgt : d[v + 1];
                float *hs = h[s];
                const SiteQ q = site_quantities(hs[1], hs[2], hs[3], hs[4], hs[5], hs[6], hs[7],
                                                hs[8], d[v], dxm, dxp,
                                                GR ? d[v] : (swap_y ? dyp[v] : dym[v]),
                                                swap_y ? dym[v] : dyp[v], c,
                                                GR ? __fmul_rn(2.f, a15v[v]) : a15v[v]);
                float o[9];
                o[0] = __fmaf_rn(c.om1, hs[0], q.wB);                           // rest
                pair_out(hs[1], hs[3], q.jx, q.ux, q.Ax, q.wB, c, o[1], o[3]);  // e = (1, 0)
                pair_out(hs[2], hs[4], q.jy, q.uy, q.Ay, q.wB, c, o[2], o[4]);  // e = (0, 1)
                pair_out(hs[5], hs[7], __fadd_rn(q.jx, q.jy), __fadd_rn(q.ux, q.uy),
                         __fadd_rn(q.Ax, q.Ay), q.wB, c, o[5], o[7]);  // e = (1, 1)
                pair_out(hs[6], hs[8], __fsub_rn(q.jy, q.jx), __fsub_rn(q.uy, q.ux),
                         __fsub_rn(q.Ay, q.Ax), q.wB, c, o[6], o[8]);  // e = (-1, 1)
#pragma unroll
                for (int i = 0; i < 9; ++i) hs[i] = o[i];
            }
            pack_sites(w, v0, h, r);
        }
        if (!act || !keep) return;
        const size_t row = (size_t)r * nx + xs;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const size_t idx = (size_t)i * P + row;
            if (VSS_IN_BOUNDS(idx, V, 9 * P)) store_words<S, V>(fout + idx, w[i]);
        }
    }

    // Advances rows y0 .. y1-1 (0 <= y0 < y1 <= ny) by one step, walking
    // down (dir = +1, rows in increasing y) or up (dir = -1).  The direction
    // changes only the order of the rows, not any result.  The walk pulls
    // n + 2 rows (one beyond each end of the segment, for drho only) and
    // collides the row before the one just pulled.
    __device__ __forceinline__ void run(int y0, int y1, int dir, const Coef &c) const {
        // Pulled-row cursor q and its source rows q-1, q+1, all wrapped.
        int q0 = dir > 0 ? ((y0 == 0) ? ny - 1 : y0 - 1) : (y1 == ny ? 0 : y1);
        int qm = (q0 == 0) ? ny - 1 : q0 - 1;
        int qp = (q0 + 1 == ny) ? 0 : q0 + 1;

        uint32_t wc[9][NW], wn[9][NW];
        float d2[V], d1[V], d0[V];  // drho of the rows pulled two, one and zero pulls ago
        float l1 = 0.f, r1 = 0.f, l0, r0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            d2[v] = 0.f;
            d1[v] = 0.f;
        }
        const int n = y1 - y0;
        for (int k = 0; k < n + 2; ++k) {
            pull_row(qm, q0, qp, wn, d0, l0, r0);
            if (k >= 2) {
                const int r = dir > 0 ? y0 + (k - 2) : y1 - 1 - (k - 2);
                if (dir > 0)
                    collide_store(r, wc, d1, d2, d0, l1, r1, c);
                else
                    collide_store(r, wc, d1, d0, d2, l1, r1, c);
            }
#pragma unroll
            for (int i = 0; i < 9; ++i)
#pragma unroll
                for (int kk = 0; kk < NW; ++kk) wc[i][kk] = wn[i][kk];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                d2[v] = d1[v];
                d1[v] = d0[v];
            }
            l1 = l0;
            r1 = r0;
            advance(qm, q0, qp, dir);
        }
    }

    // Asynchronous copy (cp.async, through L2 only) of this lane's nine
    // 16-byte vectors of pulled row q0 into `slot` ([9][32] vectors), as one
    // commit group.  Same sources as load_row.
    __device__ __forceinline__ void issue_row_async(int qm, int q0, int qp, uint4 *slot) const {
        const int xl = act ? xs : x0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sr = (EYi(i) > 0) ? qm : ((EYi(i) < 0) ? qp : q0);
            const size_t idx = (size_t)i * P + (size_t)sr * nx + xl;
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(slot + i * 32 + lane);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(fin + idx)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // The helper lane's value of pulled row q0 (see load_row).
    __device__ __forceinline__ uint32_t load_helper(int qm, int q0, int qp) const {
        const int gsr = (gey > 0) ? qm : ((gey < 0) ? qp : q0);
        const size_t gidx = (size_t)gdir * P + (size_t)gsr * nx + gcol;
        return load_elem<S, LD>(fin + gidx);
    }
    // Split walk: the value of the lane's right-side role.
    __device__ __forceinline__ uint32_t load_helper2(int qm, int q0, int qp) const {
        const int gsr = (gey2 > 0) ? qm : ((gey2 < 0) ? qp : q0);
        const size_t gidx = (size_t)gdir2 * P + (size_t)gsr * nx + gcol2;
        return load_elem<S, LD>(fin + gidx);
    }

    // As run(), with the rows moved through shared memory so that one row of
    // loads is in flight while the warp computes, without holding it in
    // registers (8-site 16-bit lanes, 128-bit vectors, NW == 4).  `buf` is the
    // warp's [2][9][32] 16-byte vectors: a landing slot for the row being
    // copied and a stash for the pulled row waiting to be collided.  Row k+1
    // is copied while row k is finished and row k-1 collided; the copy into
    // the landing slot is issued only after the words read from it have been
    // used (the shuffles of finish_pull), so it cannot overwrite them first.
    // A lane reads only what it copied or wrote.
    __device__ __forceinline__ void run_async(int y0, int y1, int dir, const Coef &c,
                                              uint4 *buf) const {
        static_assert(NW == 4, "the row buffers hold four words per lane and direction");
        uint4 *land = buf;
        uint4 *stash = buf + 9 * 32;
        // c2 field: two slots of the lane's eight 1.5-alpha values ([2][32]
        // 16-byte vectors each) after the stash.  The values a row's collision
        // needs are copied with the pulled row before it, in the same commit
        // group, into the slot the previous collision did not read.
        uint4 *aslots = buf + 18 * 32;
        (void)aslots;
        int q0 = dir > 0 ? ((y0 == 0) ? ny - 1 : y0 - 1) : (y1 == ny ? 0 : y1);
        int qm = (q0 == 0) ? ny - 1 : q0 - 1;
        int qp = (q0 + 1 == ny) ? 0 : q0 + 1;

        float d2[V], d1[V], d0[V];
        float l1 = 0.f, r1 = 0.f, l0, r0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            d2[v] = 0.f;
            d1[v] = 0.f;
        }
        const int n = y1 - y0;
        const int K = n + 2;
        issue_row_async(qm, q0, qp, land);
        uint32_t gnext = load_helper(qm, q0, qp);
        for (int k = 0; k < K; ++k) {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            uint32_t w[9][NW];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const uint4 u = land[i * 32 + lane];
                w[i][0] = u.x;
                w[i][1] = u.y;
                w[i][2] = u.z;
                w[i][3] = u.w;
            }
            const uint32_t g = gnext;
            advance(qm, q0, qp, dir);
            finish_pull(w, g, d0, l0, r0);
            if (k + 1 < K) {
                if constexpr (VA) {
                    if (k >= 1) {
                        // alpha of the row collided at k + 1 (segment row k - 1)
                        const int ra = dir > 0 ? y0 + (k - 1) : y1 - 1 - (k - 1);
                        const float *src = a15f + (size_t)ra * nx + (act ? xs : x0);
                        uint4 *dst = aslots + ((k + 1) & 1) * 64 + lane;
#pragma unroll
                        for (int h = 0; h < 2; ++h)
                            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                                             (uint32_t)__cvta_generic_to_shared(dst + h * 32)),
                                         "l"(src + 4 * h)
                                         : "memory");
                    }
                }
                issue_row_async(qm, q0, qp, land);
                gnext = load_helper(qm, q0, qp);
            }
            if (k >= 2) {
                uint32_t wc[9][NW];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const uint4 u = stash[i * 32 + lane];
                    wc[i][0] = u.x;
                    wc[i][1] = u.y;
                    wc[i][2] = u.z;
                    wc[i][3] = u.w;
                    stash[i * 32 + lane] = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
                }
                const int r = dir > 0 ? y0 + (k - 2) : y1 - 1 - (k - 2);
                const uint4 *as = VA ? aslots + (k & 1) * 64 : nullptr;
                if (dir > 0)
                    collide_store(r, wc, d1, d2, d0, l1, r1, c, true, false, as);
                else
                    collide_store(r, wc, d1, d0, d2, l1, r1, c, true, false, as);
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    stash[i * 32 + lane] = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                d2[v] = d1[v];
                d1[v] = d0[v];
            }
            l1 = l0;
            r1 = r0;
        }
    }

    // run_async for the split walk (SEG == 16): y0, y1 and dir are the
    // lane's half's segment; K is the larger half's row count plus two, the
    // pulls both halves make.  The shorter half pulls rows past its segment
    // (wrapped, so in range) and stores none of them.  The rows differ
    // between the halves, so they are per-lane values here: only the pulled
    // row q is kept (its neighbours and the collided row are derived from it).
    __device__ __forceinline__ void run_async_split(int y0, int y1, int dir, int K,
                                                    const Coef &c, uint4 *buf) const {
        static_assert(NW == 4 && SEG == 16, "8-site 16-bit split walk");
        uint4 *land = buf;
        uint4 *stash = buf + 9 * 32;
        const int n = y1 - y0;
        int q = dir > 0 ? ((y0 == 0) ? ny - 1 : y0 - 1) : (y1 == ny ? 0 : y1);

        float d2[V], d1[V], d0[V];
        float l1 = 0.f, r1 = 0.f, l0, r0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            d2[v] = 0.f;
            d1[v] = 0.f;
        }
        uint32_t gnext, gnext2;
        {
            const int qm = (q == 0) ? ny - 1 : q - 1, qp = (q + 1 == ny) ? 0 : q + 1;
            issue_row_async(qm, q, qp, land);
            gnext = load_helper(qm, q, qp);
            gnext2 = load_helper2(qm, q, qp);
        }
        for (int k = 0; k < K; ++k) {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            uint32_t w[9][NW];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const uint4 u = land[i * 32 + lane];
                w[i][0] = u.x;
                w[i][1] = u.y;
                w[i][2] = u.z;
                w[i][3] = u.w;
            }
            const uint32_t g = gnext, g2 = gnext2;
            q += dir;
            if (q < 0) q += ny;
            if (q >= ny) q -= ny;
            finish_pull(w, g, d0, l0, r0, g2);
            if (k + 1 < K) {
                const int qm = (q == 0) ? ny - 1 : q - 1, qp = (q + 1 == ny) ? 0 : q + 1;
                issue_row_async(qm, q, qp, land);
                gnext = load_helper(qm, q, qp);
                gnext2 = load_helper2(qm, q, qp);
            }
            if (k >= 2) {
                uint32_t wc[9][NW];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const uint4 u = stash[i * 32 + lane];
                    wc[i][0] = u.x;
                    wc[i][1] = u.y;
                    wc[i][2] = u.z;
                    wc[i][3] = u.w;
                    stash[i * 32 + lane] = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
                }
                // The collided row was pulled two rows before the next one, q.
                int r = q - 2 * dir;
                if (r < 0) r += ny;
                if (r >= ny) r -= ny;
                collide_store(r, wc, d1, d2, d0, l1, r1, c, k - 2 < n, dir < 0);
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    stash[i * 32 + lane] = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
            }
#pragma unroll
            for (int v = 0; v < V; ++v) {
                d2[v] = d1[v];
                d1[v] = d0[v];
            }
            l1 = l0;
            r1 = r0;
        }
    }

    // As run(), with the loads of the next pulled row issued before the
    // current row is finished and the row before it collided, so that every
    // warp keeps one row of loads in flight while it computes.  Needs a third
    // row of registers: used with 64-bit vectors (vec 2 FP32, vec 4 16-bit).
    __device__ __forceinline__ void run_prefetch(int y0, int y1, int dir, const Coef &c) const {
        int q0 = dir > 0 ? ((y0 == 0) ? ny - 1 : y0 - 1) : (y1 == ny ? 0 : y1);
        int qm = (q0 == 0) ? ny - 1 : q0 - 1;
        int qp = (q0 + 1 == ny) ? 0 : q0 + 1;

        uint32_t wc[9][NW], wn[9][NW], wf[9][NW];
        uint32_t gn, gf;
        float d2[V], d1[V], d0[V];
        float l1 = 0.f, r1 = 0.f, l0, r0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            d2[v] = 0.f;
            d1[v] = 0.f;
        }
        const int n = y1 - y0;
        const int K = n + 2;
        load_row(qm, q0, qp, wn, gn);
        for (int k = 0; k < K; ++k) {
            advance(qm, q0, qp, dir);
            if (k + 1 < K) load_row(qm, q0, qp, wf, gf);
            finish_pull(wn, gn, d0, l0, r0);
            if (k >= 2) {
                const int r = dir > 0 ? y0 + (k - 2) : y1 - 1 - (k - 2);
                if (dir > 0)
                    collide_store(r, wc, d1, d2, d0, l1, r1, c);
                else
                    collide_store(r, wc, d1, d0, d2, l1, r1, c);
            }
#pragma unroll
            for (int i = 0; i < 9; ++i)
#pragma unroll
                for (int kk = 0; kk < NW; ++kk) {
                    wc[i][kk] = wn[i][kk];
                    wn[i][kk] = wf[i][kk];
                }
            gn = gf;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                d2[v] = d1[v];
                d1[v] = d0[v];
            }
            l1 = l0;
            r1 = r0;
        }
    }

    // The same walk with two rows of loads in flight ahead of the row being
    // pulled (one more row of raw words in registers): for kernels run at
    // lower occupancy, where one row per warp leaves too few bytes in flight.
    __device__ __forceinline__ void run_prefetch2(int y0, int y1, int dir, const Coef &c) const {
        int q0 = dir > 0 ? ((y0 == 0) ? ny - 1 : y0 - 1) : (y1 == ny ? 0 : y1);
        int qm = (q0 == 0) ? ny - 1 : q0 - 1;
        int qp = (q0 + 1 == ny) ? 0 : q0 + 1;

        uint32_t wc[9][NW], wn[9][NW], wf[9][NW], wg[9][NW];
        uint32_t gn, gf, gg;
        float d2[V], d1[V], d0[V];
        float l1 = 0.f, r1 = 0.f, l0, r0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            d2[v] = 0.f;
            d1[v] = 0.f;
        }
        const int n = y1 - y0;
        const int K = n + 2;  // K >= 3: every tile has at least one row
        load_row(qm, q0, qp, wn, gn);
        advance(qm, q0, qp, dir);
        load_row(qm, q0, qp, wf, gf);
        for (int k = 0; k < K; ++k) {
            advance(qm, q0, qp, dir);
            if (k + 2 < K) load_row(qm, q0, qp, wg, gg);
            finish_pull(wn, gn, d0, l0, r0);
            if (k >= 2) {
                const int r = dir > 0 ? y0 + (k - 2) : y1 - 1 - (k - 2);
                if (dir > 0)
                    collide_store(r, wc, d1, d2, d0, l1, r1, c);
                else
                    collide_store(r, wc, d1, d0, d2, l1, r1, c);
            }
#pragma unroll
            for (int i = 0; i < 9; ++i)
#pragma unroll
                for (int kk = 0; kk < NW; ++kk) {
                    wc[i][kk] = wn[i][kk];
                    wn[i][kk] = wf[i][kk];
                    wf[i][kk] = wg[i][kk];
                }
            gn = gf;
            gf = gg;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                d2[v] = d1[v];
                d1[v] = d0[v];
            }
            l1 = l0;
            r1 = r0;
        }
    }

    __device__ __forceinline__ void advance(int &qm, int &q0, int &qp, int dir) const {
        if (dir > 0) {
            qm = q0;
            q0 = qp;
            qp = (qp + 1 == ny) ? 0 : qp + 1;
        } else {
            qp = q0;
            q0 = qm;
            qm = (qm == 0) ? ny - 1 : qm - 1;
        }
    }
};

// ---------------------------------------------------------------------------
// Asynchronous row pipeline.  Each warp streams the rows its walk needs into a
// ring of NST shared-memory stages with bulk copies (cp.async.bulk, the TMA
// engine, no tensor map: every stage row is one to three contiguous pieces of
// a plane row), one mbarrier per stage.  A stage row holds the strip's columns
// plus PAD = 16 bytes of elements on each side (x0-PAD .. x0+wa+PAD-1, wrapped),
// which covers the shifted pulls and both halo sites, so all reads of a row
// come from shared memory.  The warp keeps NST-1 rows in flight ahead of the
// row it is pulling: the loads no longer wait in registers, and the number of
// bytes in flight is set by the stage count instead of by occupancy.  The
// arithmetic is the Walker's (finish_pull, collide_store): results are bitwise
// the same as the register walk.

constexpr int STATUS_TIMEOUT = -5;  // written to the status word when a wait runs out

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint32_t bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    // The suspend-time hint (ns) lets the thread sleep until the phase
    // completes instead of spinning and taking issue slots from other warps.
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(1000000u)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                              uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Waits for phase `parity` of barrier `bar` with a wall-clock limit; every
// lane polls, and the warp agrees on the outcome.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  unsigned long long limit_ns) {
    bool ok = mbar_try_wait(bar, parity);
    if (!__all_sync(FULL, ok)) {
        const unsigned long long t0 = globaltimer_ns();
        while (!ok) {
            ok = mbar_try_wait(bar, parity);
            if (!ok && globaltimer_ns() - t0 > limit_ns) break;
        }
    }
    return __all_sync(FULL, ok);
}

template <int S>
struct TmaGeom {
    static constexpr int V = (S == ST_F32) ? 4 : 8;  // 16 bytes of elements per lane
    static constexpr int EB = (S == ST_F32) ? 4 : 2;
    static constexpr int PAD = 16 / EB;
    static constexpr int RW = 32 * V + 2 * PAD;  // elements per stage row
    static constexpr int RWB = RW * EB;          // 544 bytes
    static constexpr int STAGE_B = 9 * RWB;      // nine directions
};

// Dynamic shared memory of a block of `warps` warps with NST stages each.
__host__ __device__ constexpr int tma_bar_bytes(int warps, int nst) {
    return ((warps * nst * 8) + 127) / 128 * 128;
}
template <int S>
__host__ __device__ constexpr int tma_smem_bytes(int warps, int nst) {
    return tma_bar_bytes(warps, nst) + warps * nst * TmaGeom<S>::STAGE_B;
}

template <int S, int NST>
struct TmaWalker {
    using G = TmaGeom<S>;
    static constexpr int V = G::V;
    static constexpr int EB = G::EB;
    static constexpr int PAD = G::PAD;
    static constexpr int NW = Pack<S, V>::NW;
    using Wk = Walker<S, V, LD_NC>;

    Wk wk;
    unsigned char *stages;  // NST * STAGE_B bytes
    uint32_t bars;          // NST mbarriers, 8 bytes apart
    // pieces of a stage row: source column, stage offset and length (elements)
    int ps0, pc0;            // left wrap piece (stage offset 0)
    int ps1, pd1, pc1;       // main piece
    int pd2, pc2;            // right wrap piece (source column 0)
    uint32_t stage_tx;      // bytes one stage receives
    unsigned long long limit_ns;

    __device__ __forceinline__ TmaWalker(const void *fin, void *fout, int nx, int ny, size_t P,
                                         int x0, unsigned char *stages_, uint32_t bars_,
                                         unsigned long long limit)
        : wk(fin, fout, nx, ny, P, x0), stages(stages_), bars(bars_), limit_ns(limit) {
        // Columns x0-PAD .. x0+wa+PAD-1 in three wrapped pieces (left wrap,
        // main, right wrap; the wrap pieces are empty away from the grid's
        // edges).  With nx a multiple of V (>= PAD) every piece starts and ends
        // on 16 bytes.  Fixed slots keep the pieces in registers.
        const int lo = x0 - PAD, hi = x0 + wk.wa + PAD;
        const int mlo = lo < 0 ? 0 : lo;
        const int mhi = hi < nx ? hi : nx;
        ps0 = nx + lo;  // left wrap: columns nx-PAD .. nx-1 (used when lo < 0)
        pc0 = lo < 0 ? -lo : 0;
        ps1 = mlo;
        pd1 = mlo - lo;
        pc1 = mhi - mlo;
        pd2 = mhi - lo;  // right wrap: columns 0 .. PAD-1 (used when hi > nx)
        pc2 = hi > nx ? hi - nx : 0;
        stage_tx = 9u * (uint32_t)(wk.wa + 2 * PAD) * EB;
    }

    __device__ __forceinline__ uint32_t bar(int s) const { return bars + 8u * s; }

    // Starts the copies of pulled row index k (row q) into stage k % NST.
    // Lane 0 announces the bytes; lanes 0..8 copy direction i = lane.
    __device__ __forceinline__ void issue(int k, int q) const {
        const int s = k % NST;
        const uint32_t b = bar(s);
        if (wk.lane == 0) mbar_arrive_expect_tx(b, stage_tx);
        __syncwarp();
        if (wk.lane < 9) {
            const int i = wk.lane;
            int sr = q - EYi(i);
            if (sr < 0) sr += wk.ny;
            if (sr >= wk.ny) sr -= wk.ny;
            const unsigned char *src =
                reinterpret_cast<const unsigned char *>(wk.fin) +
                ((size_t)i * wk.P + (size_t)sr * wk.nx) * EB;
            const uint32_t dst = smem_u32(stages + (size_t)s * G::STAGE_B + (size_t)i * G::RWB);
            fence_proxy_async_smem();
            if (pc0) bulk_copy_g2s(dst, src + (size_t)ps0 * EB, (uint32_t)pc0 * EB, b);
            bulk_copy_g2s(dst + pd1 * EB, src + (size_t)ps1 * EB, (uint32_t)pc1 * EB, b);
            if (pc2) bulk_copy_g2s(dst + pd2 * EB, src, (uint32_t)pc2 * EB, b);
        }
    }

    // Reads the lane's words and helper value of row index k from its stage.
    __device__ __forceinline__ void read(int k, uint32_t (&w)[9][NW], uint32_t &g) const {
        const unsigned char *st = stages + (size_t)(k % NST) * G::STAGE_B;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (wk.act) {
                const unsigned char *p = st + i * G::RWB + (PAD + wk.lane * V) * EB;
                uint4 r = *reinterpret_cast<const uint4 *>(p);
                w[i][0] = r.x;
                w[i][1] = r.y;
                w[i][2] = r.z;
                w[i][3] = r.w;
            } else {
#pragma unroll
                for (int kk = 0; kk < NW; ++kk) w[i][kk] = 0u;
            }
        }
        {
            const unsigned char *p = st + wk.gdir * G::RWB + (PAD + wk.goff) * EB;
            if constexpr (S == ST_F32)
                g = *reinterpret_cast<const uint32_t *>(p);
            else
                g = (uint32_t) * reinterpret_cast<const unsigned short *>(p);
        }
    }

    // Waits for row index k; on a timeout records it, waits (bounded) for the
    // copies still in flight and reports failure.
    __device__ __forceinline__ bool wait_row(int k, int issued, int *status) const {
        if (mbar_wait_bounded(bar(k % NST), (uint32_t)((k / NST) & 1), limit_ns)) return true;
        if (wk.lane == 0) atomicCAS(status, 0, STATUS_TIMEOUT);
        for (int kk = k; kk < issued; ++kk)
            mbar_wait_bounded(bar(kk % NST), (uint32_t)((kk / NST) & 1), limit_ns);
        return false;
    }

    __device__ __forceinline__ void run(int y0, int y1, int dir, const Coef &c, int *status) {
        const int ny = wk.ny;
        if (wk.lane == 0) {
            for (int s = 0; s < NST; ++s) mbar_init(bar(s), 1);
            fence_mbar_init();
        }
        __syncwarp();
        const int n = y1 - y0;
        const int K = n + 2;  // pulled rows: one beyond each end of the segment
        int q = dir > 0 ? ((y0 == 0) ? ny - 1 : y0 - 1) : (y1 == ny ? 0 : y1);
        // Issue the first NST rows; qi / ki track the next row to issue.
        int qi = q, ki = 0;
        for (; ki < NST && ki < K; ++ki) {
            issue(ki, qi);
            qi += dir;
            if (qi < 0) qi += ny;
            if (qi >= ny) qi -= ny;
        }
        uint32_t wc[9][NW], wn[9][NW];
        float dprev[V], dcur[V], dnext[V];
        float dlc, drc, dln, drn;
        uint32_t g;
        bool ok = true;
        // Row index 0: drho only.  Row index 1: the first row of the segment.
        ok = wait_row(0, ki, status);
        if (ok) {
            read(0, wn, g);
            wk.finish_pull(wn, g, dprev, dln, drn);
            __syncwarp();
            if (ki < K) {
                issue(ki, qi);
                ++ki;
                qi += dir;
                if (qi < 0) qi += ny;
                if (qi >= ny) qi -= ny;
            }
            ok = wait_row(1, ki, status);
        }
        if (ok) {
            read(1, wc, g);
            wk.finish_pull(wc, g, dcur, dlc, drc);
            __syncwarp();
            if (ki < K) {
                issue(ki, qi);
                ++ki;
                qi += dir;
                if (qi < 0) qi += ny;
                if (qi >= ny) qi -= ny;
            }
        }
        for (int k = 0; ok && k < n; ++k) {
            const int r = dir > 0 ? y0 + k : y1 - 1 - k;
            ok = wait_row(k + 2, ki, status);
            if (!ok) break;
            read(k + 2, wn, g);
            wk.finish_pull(wn, g, dnext, dln, drn);
            __syncwarp();
            if (ki < K) {
                issue(ki, qi);
                ++ki;
                qi += dir;
                if (qi < 0) qi += ny;
                if (qi >= ny) qi -= ny;
            }
            if (dir > 0)
                wk.collide_store(r, wc, dcur, dprev, dnext, dlc, drc, c);
            else
                wk.collide_store(r, wc, dcur, dnext, dprev, dlc, drc, c);
#pragma unroll
            for (int i = 0; i < 9; ++i)
#pragma unroll
                for (int kk = 0; kk < NW; ++kk) wc[i][kk] = wn[i][kk];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                dprev[v] = dcur[v];
                dcur[v] = dnext[v];
            }
            dlc = dln;
            drc = drn;
        }
        __syncwarp();
        if (ok && wk.lane == 0)
            for (int s = 0; s < NST; ++s) mbar_inval(bar(s));
    }
};

}  // namespace vss
