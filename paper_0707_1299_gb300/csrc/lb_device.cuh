// lb_device.cuh -- device-side building blocks of the forced D3Q19 MRT
// lattice Boltzmann kernels: storage conversion, pull streaming of one
// site, the moment-space collision with forcing, and Peskin's kernel.
//
// Population i of site (x, y, z) lives at  buf[i * V + (z * ny + y) * nx + x]
// (structure of arrays), as the deviation df = fbar - w_i from the rest
// state.  Velocity order (the C ABI's):
//   0 (0,0,0)  1 (1,0,0)  2 (-1,0,0)  3 (0,1,0)  4 (0,-1,0)  5 (0,0,1)
//   6 (0,0,-1) 7 (1,1,0)  8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0) 11 (1,0,1)
//   12 (-1,0,-1) 13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1) 16 (0,-1,-1)
//   17 (0,1,-1) 18 (0,-1,1)
#pragma once

#include <cuda_bf16.h>
#include <type_traits>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace lbk {

constexpr int NQ = 19;
constexpr int TILE_X = 32;  // one warp of x-consecutive sites = one force tile

// Lattice geometry, passed by value to every kernel.  Site indices are
// 32-bit: the C ABI keeps nx * ny * nz below 2^32.
struct Geom {
    int nx, ny, nz;
    int ntx;            // tiles per x-row: ceil(nx / 32)
    unsigned plane;     // nx * ny
    long long V;        // nx * ny * nz
    long long ntiles;   // ntx * ny * nz
    int wall_lo, wall_hi;  // solid z-planes, -1 = none
};

__device__ __forceinline__ bool is_solid(const Geom& g, int z) {
    return z == g.wall_lo || z == g.wall_hi;
}

// Force flags.  Spreading sets the byte flag of every 8-site x-group it adds
// force to (a plain store: any number of writers store the same value); the
// four groups of a 32-site x-row tile form one 32-bit word, read once per
// warp, byte lane / 8 for lane.  The collide kernel reads the field only in
// flagged groups; where the field is spread anew every step (mobile
// colloids, batches) it also writes the velocity there and then zeroes the
// consumed field and the flags.
using flag_t = unsigned char;
constexpr int GROUP_X = 8;  // sites of an x-group

// This lane's group flag in a tile's flag word (x the lane's site offset in the tile).
__device__ __forceinline__ unsigned group_flag(unsigned word, unsigned x_in_tile) {
    return (word >> (8u * (x_in_tile / GROUP_X))) & 0xFFu;
}

// Force and velocity fields: FIELD_W elements of the arithmetic type a site,
// x, y, z and an unused fourth (kept zero), so that a node's three
// components are one 16-byte word in float: the spread adds a node with one
// vector reduction, the interpolation reads it with one load.  field_ldg
// reads through the read-only path (see reset_group_flag), field_ld with a
// plain load; field_st writes (zero in the fourth element), field_add adds.
constexpr int FIELD_W = 4;
__device__ __forceinline__ void field_ldg(const float* f, size_t site, float& x, float& y, float& z) {
    const float4 q = __ldg((const float4*)f + site);
    x = q.x, y = q.y, z = q.z;
}
__device__ __forceinline__ void field_ldg(const double* f, size_t site, double& x, double& y, double& z) {
    const double2 q = __ldg((const double2*)(f + FIELD_W * site));
    x = q.x, y = q.y, z = __ldg(f + FIELD_W * site + 2);
}
__device__ __forceinline__ void field_ld(const float* f, size_t site, float& x, float& y, float& z) {
    const float4 q = *((const float4*)f + site);
    x = q.x, y = q.y, z = q.z;
}
__device__ __forceinline__ void field_ld(const double* f, size_t site, double& x, double& y, double& z) {
    const double2 q = *(const double2*)(f + FIELD_W * site);
    x = q.x, y = q.y, z = f[FIELD_W * site + 2];
}
__device__ __forceinline__ void field_st(float* f, size_t site, float x, float y, float z) {
    *((float4*)f + site) = make_float4(x, y, z, 0.0f);
}
__device__ __forceinline__ void field_st(double* f, size_t site, double x, double y, double z) {
    *(double2*)(f + FIELD_W * site) = make_double2(x, y);
    *(double2*)(f + FIELD_W * site + 2) = make_double2(z, 0.0);
}
__device__ __forceinline__ void field_add(float* f, size_t site, float x, float y, float z) {
    const size_t a = __cvta_generic_to_global((float4*)f + site);
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(a), "f"(x), "f"(y), "f"(z), "f"(0.0f)
                 : "memory");
}
__device__ __forceinline__ void field_add(double* f, size_t site, double x, double y, double z) {
    atomicAdd(f + FIELD_W * site, x);
    atomicAdd(f + FIELD_W * site + 1, y);
    atomicAdd(f + FIELD_W * site + 2, z);
}

// ----------------------------------------------------------- storage types
// df is stored as S and handled in arithmetic type T.  The half-precision
// formats store df * scale (a power of two) to keep df out of subnormals.
template <typename S> struct Store;
// ld/st move the stored number without any scaling: for the half format
// that is df * scale, and the kernels either work in those scaled units
// (k_collide) or multiply by 1 / scale themselves.  st takes 32 random
// bits `rnd`, used only by the 16-bit formats, which round stochastically:
// a per-step change far below one unit in the last place would otherwise be
// rounded away the same way every step.
template <> struct Store<double> {
    using T = double;
    static constexpr bool kCompensate = false;  // FP64 needs no compensated momentum sum
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ double ld(const double* p, unsigned i) { return __ldg(p + i); }
    static __device__ __forceinline__ void st(double* p, unsigned i, double v, unsigned) { __stcs(p + i, v); }
};
template <> struct Store<float> {
    using T = float;
    static constexpr bool kCompensate = true;
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ float ld(const float* p, unsigned i) { return __ldg(p + i); }
    static __device__ __forceinline__ void st(float* p, unsigned i, float v, unsigned) { __stcs(p + i, v); }
};
template <> struct Store<__half> {
    using T = float;
    static constexpr bool kCompensate = false;  // storage rounding dominates
    static constexpr bool kScaled = true;
    static __device__ __forceinline__ float ld(const __half* p, unsigned i) { return __half2float(__ldg(p + i)); }
    // Stochastic rounding to half: add 13 random bits below the 10-bit half
    // mantissa to the float's magnitude, then truncate.  Values beyond the
    // half range saturate to +-65504.
    static __device__ __forceinline__ unsigned short bits(float v, unsigned rnd) {
        const unsigned b = __float_as_uint(v) + (rnd >> 19);
        return __half_as_ushort(__float2half_rz(__uint_as_float(b)));
    }
    static __device__ __forceinline__ void st(__half* p, unsigned i, float v, unsigned rnd) {
        p[i] = __ushort_as_half(bits(v, rnd));
    }
    // both elements of a word
    static __device__ __forceinline__ float2 unpack2(unsigned w) {
        __half2 h;
        memcpy(&h, &w, sizeof(w));
        return __half22float2(h);
    }
    // stochastic rounding of two values into one word by the conversion's
    // own stochastic-rounding mode (sm_100a and later): random bits 12:0 of
    // rb dither lo, bits 28:16 hi; beyond the half range the result is
    // infinite (and caught by the finiteness checks)
    static __device__ __forceinline__ unsigned bits2_rs(float lo, float hi, unsigned rb) {
        unsigned r;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(r) : "f"(hi), "f"(lo), "r"(rb));
        return r;
    }
};
template <> struct Store<__nv_bfloat16> {
    using T = float;
    static constexpr bool kCompensate = false;
    static constexpr bool kScaled = false;  // bfloat16 has the float exponent range
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p, unsigned i) {
        return __bfloat162float(__ldg(p + i));
    }
    // Stochastic rounding to bfloat16: add 16 random bits to the dropped half
    // of the float, keep the upper half.
    static __device__ __forceinline__ unsigned short bits(float v, unsigned rnd) {
        return (unsigned short)((__float_as_uint(v) + (rnd >> 16)) >> 16);
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, unsigned i, float v, unsigned rnd) {
        p[i] = __ushort_as_bfloat16(bits(v, rnd));
    }
    static __device__ __forceinline__ float2 unpack2(unsigned w) {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
    }
    // as Store<__half>::bits2_rs: random bits 15:0 dither lo, 31:16 hi
    static __device__ __forceinline__ unsigned bits2_rs(float lo, float hi, unsigned rb) {
        unsigned r;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(r) : "f"(hi), "f"(lo), "r"(rb));
        return r;
    }
};

// Counter-based random bits for stochastic rounding: a hash of the site and
// the step seeds a linear congruential sequence, one draw per population.
__device__ __forceinline__ unsigned rng_seed(unsigned site, unsigned step_seed) {
    unsigned x = site * 0x9E3779B9u ^ step_seed;
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ unsigned rng_next(unsigned& x) {
    x = x * 1664525u + 1013904223u;
    return x;
}
// One draw for the two 16-bit halves of a stochastically rounded word: the
// high half of the state is its well-mixed part, so it goes to both halves
// (folded into the low one, whose own low bits have short periods).
__device__ __forceinline__ unsigned rng_next2(unsigned& x) {
    const unsigned r = rng_next(x);
    return r ^ (r >> 16);
}

// ------------------------------------------------------------ pull stream
// The 19 population arrays, one pointer each (kernel parameter space), so
// that every load or store needs one 32-bit index and no 64-bit i * V.
template <typename S>
struct Pops {
    S* p[NQ];
};

// Site offsets of the neighbours of (x, y, z), periodic, in unsigned
// 32-bit arithmetic (differences wrap modulo 2^32 and add back exactly).
struct Nbr {
    unsigned c;              // (z * ny + y) * nx: row of the site
    unsigned dym, dyp;       // row(y -+ 1) - row(y)
    unsigned dzm, dzp;       // row(z -+ 1) - row(z)
    unsigned x, xm, xp;
    bool solid_zm, solid_zp;
};

__device__ __forceinline__ Nbr neighbours(const Geom& g, int x, int y, int z) {
    Nbr n;
    const unsigned nx = (unsigned)g.nx;
    n.c = (unsigned)z * g.plane + (unsigned)y * nx;
    n.dym = (y == 0) ? (unsigned)(g.ny - 1) * nx : 0u - nx;
    n.dyp = (y == g.ny - 1) ? 0u - (unsigned)(g.ny - 1) * nx : nx;
    n.dzm = (z == 0) ? (unsigned)(g.nz - 1) * g.plane : 0u - g.plane;
    n.dzp = (z == g.nz - 1) ? 0u - (unsigned)(g.nz - 1) * g.plane : g.plane;
    n.x = (unsigned)x;
    n.xm = (x == 0) ? nx - 1 : (unsigned)x - 1;
    n.xp = (x == g.nx - 1) ? 0u : (unsigned)x + 1;
    n.solid_zm = is_solid(g, z == 0 ? g.nz - 1 : z - 1);
    n.solid_zp = is_solid(g, z == g.nz - 1 ? 0 : z + 1);
    return n;
}

// df_i(x) = df*_i(x - c_i); where x - c_i is a solid node the population
// bounces back: df_i(x) = df*_ibar(x).
template <typename S, bool WALLS>
__device__ __forceinline__ void pull19(const Pops<S>& src, const Nbr& n, typename Store<S>::T f[NQ]) {
    using St = Store<S>;
    const unsigned own = n.c + n.x;
    const unsigned ym = n.c + n.dym, yp = n.c + n.dyp, zm = n.c + n.dzm, zp = n.c + n.dzp;
    f[0] = St::ld(src.p[0], own);
    f[1] = St::ld(src.p[1], n.c + n.xm);
    f[2] = St::ld(src.p[2], n.c + n.xp);
    f[3] = St::ld(src.p[3], ym + n.x);
    f[4] = St::ld(src.p[4], yp + n.x);
    f[7] = St::ld(src.p[7], ym + n.xm);
    f[8] = St::ld(src.p[8], yp + n.xp);
    f[9] = St::ld(src.p[9], yp + n.xm);
    f[10] = St::ld(src.p[10], ym + n.xp);
    if (!WALLS) {
        f[5] = St::ld(src.p[5], zm + n.x);
        f[11] = St::ld(src.p[11], zm + n.xm);
        f[14] = St::ld(src.p[14], zm + n.xp);
        f[15] = St::ld(src.p[15], zm + n.dym + n.x);
        f[18] = St::ld(src.p[18], zm + n.dyp + n.x);
        f[6] = St::ld(src.p[6], zp + n.x);
        f[12] = St::ld(src.p[12], zp + n.xp);
        f[13] = St::ld(src.p[13], zp + n.xm);
        f[16] = St::ld(src.p[16], zp + n.dyp + n.x);
        f[17] = St::ld(src.p[17], zp + n.dym + n.x);
    } else {
        // one load per population: a solid source selects the opposite
        // population of the site itself (uniform across the warp)
        const bool bm = n.solid_zm, bp = n.solid_zp;
        f[5] = St::ld(bm ? src.p[6] : src.p[5], bm ? own : zm + n.x);
        f[11] = St::ld(bm ? src.p[12] : src.p[11], bm ? own : zm + n.xm);
        f[14] = St::ld(bm ? src.p[13] : src.p[14], bm ? own : zm + n.xp);
        f[15] = St::ld(bm ? src.p[16] : src.p[15], bm ? own : zm + n.dym + n.x);
        f[18] = St::ld(bm ? src.p[17] : src.p[18], bm ? own : zm + n.dyp + n.x);
        f[6] = St::ld(bp ? src.p[5] : src.p[6], bp ? own : zp + n.x);
        f[12] = St::ld(bp ? src.p[11] : src.p[12], bp ? own : zp + n.xp);
        f[13] = St::ld(bp ? src.p[14] : src.p[13], bp ? own : zp + n.xm);
        f[16] = St::ld(bp ? src.p[15] : src.p[16], bp ? own : zp + n.dyp + n.x);
        f[17] = St::ld(bp ? src.p[18] : src.p[17], bp ? own : zp + n.dym + n.x);
    }
}

// ------------------------------------------- pull stream, two sites a thread
// The 16-bit formats with nx even: a thread takes the x-adjacent sites x0,
// x0 + 1 (x0 even), whose values of one population share a 32-bit word.
// A population pulled from x - 1 or x + 1 straddles two words: the
// neighbouring lane's word arrives by shuffle (the lane at a warp or row
// edge loads it, wrapping periodically), and a byte permute joins the
// halves.  Inactive lanes (x0 >= nx) load nothing but take part in the
// shuffles; only a lane whose neighbour is active reads the shuffled word.
template <typename S>
__device__ __forceinline__ unsigned ldw(const S* p, unsigned e) {
    return __ldg((const unsigned*)(p + e));
}

// Which neighbour word a population's pair needs: 0 none, -1 the word
// before (pulled from x - 1: c_x = +1), +1 the word after (c_x = -1).
__host__ __device__ constexpr int pair_shift(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? -1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? 1 : 0;
}

// The pulls of pull19 for the pair (x0, x0 + 1); n holds the rows of (y, z)
// (its x fields are not used).  With walls a solid source selects the
// opposite population of the site itself, unshifted (uniform per warp).
// Every load is issued first (the own-row word of each population, and the
// edge lanes' words beyond the warp), then the shuffles and permutes.
template <typename S, bool BOUNCE, typename Between>
__device__ __forceinline__ void pull19_pair_impl(const Pops<S>& src, const Nbr& n, unsigned x0, unsigned nx, int lane,
                                                 bool active, unsigned w[NQ], Between&& between) {
    const unsigned c = n.c, ym = n.c + n.dym, yp = n.c + n.dyp, zm = n.c + n.dzm, zp = n.c + n.dzp;
    const bool bm = BOUNCE && n.solid_zm, bp = BOUNCE && n.solid_zp;
    // source population and row of each pull; a bounced pull is unshifted
    const S* ptr[NQ];
    unsigned row[NQ];
    bool shifted[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        ptr[i] = src.p[i];
        shifted[i] = pair_shift(i) != 0;
    }
    row[0] = c;
    row[1] = c;
    row[2] = c;
    row[3] = ym;
    row[4] = yp;
    row[7] = ym;
    row[8] = yp;
    row[9] = yp;
    row[10] = ym;
    row[5] = zm;
    row[11] = zm;
    row[14] = zm;
    row[15] = zm + n.dym;
    row[18] = zm + n.dyp;
    row[6] = zp;
    row[12] = zp;
    row[13] = zp;
    row[16] = zp + n.dyp;
    row[17] = zp + n.dym;
    if (bm) {
        ptr[5] = src.p[6];
        ptr[11] = src.p[12];
        ptr[14] = src.p[13];
        ptr[15] = src.p[16];
        ptr[18] = src.p[17];
        row[5] = row[11] = row[14] = row[15] = row[18] = c;
        shifted[11] = shifted[14] = false;
    }
    if (bp) {
        ptr[6] = src.p[5];
        ptr[12] = src.p[11];
        ptr[13] = src.p[14];
        ptr[16] = src.p[15];
        ptr[17] = src.p[18];
        row[6] = row[12] = row[13] = row[16] = row[17] = c;
        shifted[12] = shifted[13] = false;
    }
    const bool first = lane == 0, last = lane == 31 || x0 + 2 >= nx;
    const unsigned xb = x0 == 0 ? nx - 2 : x0 - 2, xa = x0 + 2 >= nx ? 0 : x0 + 2;
    unsigned edge[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        w[i] = active ? ldw(ptr[i], row[i] + x0) : 0u;
        edge[i] = 0u;
        if (pair_shift(i) < 0 && shifted[i] && active && first) edge[i] = ldw(ptr[i], row[i] + xb);
        if (pair_shift(i) > 0 && shifted[i] && active && last) edge[i] = ldw(ptr[i], row[i] + xa);
    }
    between();  // more loads of the caller, in flight with these before the shuffles wait for them
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        if (pair_shift(i) < 0 && shifted[i]) {  // (element x0 - 1, element x0)
            unsigned prev = __shfl_up_sync(0xffffffffu, w[i], 1);
            if (first) prev = edge[i];
            w[i] = __byte_perm(prev, w[i], 0x5432);
        } else if (pair_shift(i) > 0 && shifted[i]) {  // (element x0 + 1, element x0 + 2)
            unsigned next = __shfl_down_sync(0xffffffffu, w[i], 1);
            if (last) next = edge[i];
            w[i] = __byte_perm(w[i], next, 0x5432);
        }
    }
}

// A plane next to a solid one takes the bounce-back selections; every other
// plane (uniform per warp) the plain pulls.
// `between()` runs after the loads are issued and before the shuffles that
// wait for them (the collide issues its force loads there).
template <typename S, bool WALLS, typename Between>
__device__ __forceinline__ void pull19_pair(const Pops<S>& src, const Nbr& n, unsigned x0, unsigned nx, int lane,
                                            bool active, unsigned w[NQ], Between&& between) {
    if (WALLS && (n.solid_zm || n.solid_zp)) pull19_pair_impl<S, true>(src, n, x0, nx, lane, active, w, between);
    else pull19_pair_impl<S, false>(src, n, x0, nx, lane, active, w, between);
}

// ------------------------------------------ pull stream, four sites a thread
// The 16-bit formats with nx a multiple of 4: a thread takes the sites x0 ..
// x0 + 3 (x0 a multiple of 4), whose values of one population form one
// 64-bit word (lo: x0, x0 + 1; hi: x0 + 2, x0 + 3), loaded aligned (nx % 4
// == 0 makes every population row and V multiples of 4 elements).  A pull
// from x - 1 needs element x0 - 1, the high half of the previous lane's hi
// word; a pull from x + 1 needs element x0 + 4, the low half of the next
// lane's lo word: they arrive by shuffle (the lane at a warp or row edge
// loads them, wrapping periodically) and byte permutes assemble the two
// shifted words.  Inactive lanes (x0 >= nx) load nothing but take part in
// the shuffles.  Returns the two words of each population: lo[i] for the
// sites x0, x0 + 1 and hi[i] for x0 + 2, x0 + 3.
template <typename S>
__device__ __forceinline__ uint2 ldw2(const S* p, unsigned e) {
    return __ldg((const uint2*)(p + e));
}

template <typename S, bool BOUNCE, typename Between>
__device__ __forceinline__ void pull19_quad_impl(const Pops<S>& src, const Nbr& n, unsigned x0, unsigned nx, int lane,
                                                 bool active, unsigned lo[NQ], unsigned hi[NQ], Between&& between) {
    const unsigned c = n.c, ym = n.c + n.dym, yp = n.c + n.dyp, zm = n.c + n.dzm, zp = n.c + n.dzp;
    const bool bm = BOUNCE && n.solid_zm, bp = BOUNCE && n.solid_zp;
    const S* ptr[NQ];
    unsigned row[NQ];
    bool shifted[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        ptr[i] = src.p[i];
        shifted[i] = pair_shift(i) != 0;
    }
    row[0] = c;
    row[1] = c;
    row[2] = c;
    row[3] = ym;
    row[4] = yp;
    row[7] = ym;
    row[8] = yp;
    row[9] = yp;
    row[10] = ym;
    row[5] = zm;
    row[11] = zm;
    row[14] = zm;
    row[15] = zm + n.dym;
    row[18] = zm + n.dyp;
    row[6] = zp;
    row[12] = zp;
    row[13] = zp;
    row[16] = zp + n.dyp;
    row[17] = zp + n.dym;
    if (bm) {
        ptr[5] = src.p[6];
        ptr[11] = src.p[12];
        ptr[14] = src.p[13];
        ptr[15] = src.p[16];
        ptr[18] = src.p[17];
        row[5] = row[11] = row[14] = row[15] = row[18] = c;
        shifted[11] = shifted[14] = false;
    }
    if (bp) {
        ptr[6] = src.p[5];
        ptr[12] = src.p[11];
        ptr[13] = src.p[14];
        ptr[16] = src.p[15];
        ptr[17] = src.p[18];
        row[6] = row[12] = row[13] = row[16] = row[17] = c;
        shifted[12] = shifted[13] = false;
    }
    const bool first = lane == 0, last = lane == 31 || x0 + 4 >= nx;
    // the 32-bit words holding element x0 - 1 (as its high half) and x0 + 4
    // (as its low half), wrapped periodically along the row
    const unsigned xb = x0 == 0 ? nx - 2 : x0 - 2, xa = x0 + 4 >= nx ? 0 : x0 + 4;
    uint2 w[NQ];
    unsigned edge[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        w[i] = active ? ldw2(ptr[i], row[i] + x0) : make_uint2(0u, 0u);
        edge[i] = 0u;
        if (pair_shift(i) < 0 && shifted[i] && active && first) edge[i] = ldw(ptr[i], row[i] + xb);
        if (pair_shift(i) > 0 && shifted[i] && active && last) edge[i] = ldw(ptr[i], row[i] + xa);
    }
    between();
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        if (pair_shift(i) < 0 && shifted[i]) {  // (x0 - 1, x0), (x0 + 1, x0 + 2)
            unsigned prev = __shfl_up_sync(0xffffffffu, w[i].y, 1);
            if (first) prev = edge[i];
            lo[i] = __byte_perm(prev, w[i].x, 0x5432);
            hi[i] = __byte_perm(w[i].x, w[i].y, 0x5432);
        } else if (pair_shift(i) > 0 && shifted[i]) {  // (x0 + 1, x0 + 2), (x0 + 3, x0 + 4)
            unsigned next = __shfl_down_sync(0xffffffffu, w[i].x, 1);
            if (last) next = edge[i];
            lo[i] = __byte_perm(w[i].x, w[i].y, 0x5432);
            hi[i] = __byte_perm(w[i].y, next, 0x5432);
        } else {
            lo[i] = w[i].x;
            hi[i] = w[i].y;
        }
    }
}

template <typename S, bool WALLS, typename Between>
__device__ __forceinline__ void pull19_quad(const Pops<S>& src, const Nbr& n, unsigned x0, unsigned nx, int lane,
                                            bool active, unsigned lo[NQ], unsigned hi[NQ], Between&& between) {
    if (WALLS && (n.solid_zm || n.solid_zp)) pull19_quad_impl<S, true>(src, n, x0, nx, lane, active, lo, hi, between);
    else pull19_quad_impl<S, false>(src, n, x0, nx, lane, active, lo, hi, between);
}

// Pulled populations in stored units -> df (only the half format is scaled).
template <typename S>
__device__ __forceinline__ void unscale19(typename Store<S>::T f[NQ], float inv_scale) {
    if (Store<S>::kScaled)
#pragma unroll
        for (int i = 0; i < NQ; ++i) f[i] *= inv_scale;
}

// ------------------------------------------------------------- moments
template <typename T>
struct Moments {
    T drho, jx, jy, jz;              // sum df, sum df c
    T jx_lo, jy_lo, jz_lo;           // rounding error of j (float: compensated sum; double: 0)
    T pxx, pyy, pzz, pxy, pxz, pyz;  // sum df c_a c_b
};

// s + e == a + b exactly (Knuth's two-sum; explicit round-to-nearest adds
// so that nothing is reassociated or contracted).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// Momentum j as an unevaluated sum hi + lo.  In float the rounding of
// j = sum df c would otherwise feed back into the populations every step:
// when j changes by a nearly constant increment (a uniform body force) the
// rounded increment is the same each step and the error grows linearly.
template <typename T, bool COMP> struct MomentumSum {
    static __device__ __forceinline__ void eval(const T f[NQ], Moments<T>& m) {
        const T e78 = f[7] - f[8], e910 = f[9] - f[10], e1112 = f[11] - f[12], e1314 = f[13] - f[14];
        const T e1516 = f[15] - f[16], e1718 = f[17] - f[18];
        m.jx = (f[1] - f[2]) + e78 + e910 + e1112 + e1314;
        m.jy = (f[3] - f[4]) + e78 - e910 + e1516 + e1718;
        m.jz = (f[5] - f[6]) + e1112 - e1314 + e1516 - e1718;
        m.jx_lo = m.jy_lo = m.jz_lo = T(0);
    }
};
template <> struct MomentumSum<float, true> {
    static __device__ __forceinline__ void eval(const float f[NQ], Moments<float>& m) {
        float d12, d34, d56, d78, d910, d1112, d1314, d1516, d1718;
        float r12, r34, r56, r78, r910, r1112, r1314, r1516, r1718;
        two_sum(f[1], -f[2], d12, r12);
        two_sum(f[3], -f[4], d34, r34);
        two_sum(f[5], -f[6], d56, r56);
        two_sum(f[7], -f[8], d78, r78);
        two_sum(f[9], -f[10], d910, r910);
        two_sum(f[11], -f[12], d1112, r1112);
        two_sum(f[13], -f[14], d1314, r1314);
        two_sum(f[15], -f[16], d1516, r1516);
        two_sum(f[17], -f[18], d1718, r1718);
        float s, t1, t2, t3, t4;
        // jx = d12 + d78 + d910 + d1112 + d1314
        two_sum(d12, d78, s, t1);
        two_sum(s, d910, s, t2);
        two_sum(s, d1112, s, t3);
        two_sum(s, d1314, m.jx, t4);
        m.jx_lo = ((r12 + r78) + (r910 + r1112)) + (r1314 + ((t1 + t2) + (t3 + t4)));
        // jy = d34 + d78 - d910 + d1516 + d1718
        two_sum(d34, d78, s, t1);
        two_sum(s, -d910, s, t2);
        two_sum(s, d1516, s, t3);
        two_sum(s, d1718, m.jy, t4);
        m.jy_lo = ((r34 + r78) + (r1516 - r910)) + (r1718 + ((t1 + t2) + (t3 + t4)));
        // jz = d56 + d1112 - d1314 + d1516 - d1718
        two_sum(d56, d1112, s, t1);
        two_sum(s, -d1314, s, t2);
        two_sum(s, d1516, s, t3);
        two_sum(s, -d1718, m.jz, t4);
        m.jz_lo = ((r56 + r1112) + (r1516 - r1314)) + (((t1 + t2) + (t3 + t4)) - r1718);
    }
};

template <typename T, bool COMP>
__device__ __forceinline__ Moments<T> moments19(const T f[NQ]) {
    // pair sums (c, -c); then, in FP64 (bound by its arithmetic pipe), the
    // diagonal pairs summed per plane and the diagonal second moments and
    // rho from them (22 additions); in float and the packed pair (bound by
    // bytes and issue, where the other order measured 0.6-2 % faster on
    // GB300 at 256^3) each sum written out (30 additions)
    Moments<T> m;
    const T a12 = f[1] + f[2], a34 = f[3] + f[4], a56 = f[5] + f[6];
    const T d78 = f[7] + f[8], d910 = f[9] + f[10], d1112 = f[11] + f[12], d1314 = f[13] + f[14];
    const T d1516 = f[15] + f[16], d1718 = f[17] + f[18];
    if constexpr (!std::is_same<T, double>::value) {
        m.drho = f[0] + a12 + a34 + a56 + d78 + d910 + d1112 + d1314 + d1516 + d1718;
        MomentumSum<T, COMP>::eval(f, m);
        m.pxx = a12 + d78 + d910 + d1112 + d1314;
        m.pyy = a34 + d78 + d910 + d1516 + d1718;
        m.pzz = a56 + d1112 + d1314 + d1516 + d1718;
    } else {
        const T sxy = d78 + d910, sxz = d1112 + d1314, syz = d1516 + d1718;
        MomentumSum<T, COMP>::eval(f, m);
        m.pxx = (a12 + sxy) + sxz;
        m.pyy = (a34 + sxy) + syz;
        m.pzz = (a56 + sxz) + syz;
        m.drho = ((f[0] + m.pxx) + (a34 + a56)) + syz;
    }
    m.pxy = d78 - d910;
    m.pxz = d1112 - d1314;
    m.pyz = d1516 - d1718;
    return m;
}

// Relaxation coefficients of the collision, Sec. II Eq. (fiexp) with the
// stress update read from Eq. (mrtlbe): omega = 1 / (tau + 1/2).
template <typename T>
struct Coef {
    T tau_s, tau_b, om_s, om_b;
};

// Lattice weights and Hermite coefficients rounded so that the discrete
// moment identities hold exactly for the rounded values:
//   w0 + 6 w1 + 12 w2 == 1          (mass of the reconstruction)
//   2 a1 + 8 b1 == 1                (momentum: a1 ~ 3 w1 = 1/6, b1 ~ 3 w2 = 1/12)
// Plain round-to-nearest of 1/6 gives 6 fl(1/6) = 1 + 3e-8 in float, a
// momentum gain every step that accumulates in slowly varying flows.
template <typename T> struct Wts;
template <> struct Wts<float> {
    static constexpr float w0 = 11184812.0f * 0x1p-25f;   // ~ 1/3
    static constexpr float w2 = 14913080.0f * 0x1p-29f;   // ~ 1/36
    static constexpr float w1 = 2.0f * w2;                // ~ 1/18
    static constexpr float a1 = 11184810.0f * 0x1p-26f;   // ~ 1/6
    static constexpr float b1 = 11184811.0f * 0x1p-27f;   // ~ 1/12
};
template <> struct Wts<double> {
    static constexpr double w0 = 6004799503160662.0 * 0x1p-54;
    static constexpr double w2 = 8006399337547548.0 * 0x1p-58;
    static constexpr double w1 = 2.0 * w2;
    static constexpr double a1 = 6004799503160660.0 * 0x1p-55;
    static constexpr double b1 = 6004799503160662.0 * 0x1p-56;
};

// Two sites at once on the packed FP32 datapath of sm_100 and later: F2
// holds one float of each site; every operation is the IEEE round-to-
// nearest float operation on both halves (one instruction for the pair).
// collide19 and moments19 instantiated with F2 compute two independent
// sites; products and sums are not contracted unless written as fma.
struct F2 {
    float2 v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ F2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ explicit F2(float2 a) : v(a) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(__fmul2_rn(a.v, make_float2(-1.0f, -1.0f))); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator/(F2 a, F2 b) { return F2(make_float2(a.v.x / b.v.x, a.v.y / b.v.y)); }
using ::fma;  // the float and double overloads stay visible beside F2's
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
template <> struct Wts<F2> : Wts<float> {};

// Post-collision df* from the pulled df and the local force density F:
//   A = j + F,  v = (j + F/2) / rho,  S = sum df Q,
//   X = S - rho vv,  Y = vF + Fv,
//   B = S - om_s dev(X - tau_s Y) - (om_b / 3) tr(X - tau_b Y) 1,
//   df*_i = w_i [drho + 3 A.c_i + 4.5 c_i.B.c_i - 1.5 tr B].
// Evaluation order: the momentum term 3 w_i j.c_i, the largest, enters
// last through fused multiply-adds, so it is rounded once; the force term
// 3 w_i F.c_i is added to the small terms first, so a force much smaller
// than j is not lost to the rounding of j + F.
// With SCALED, f and F are in units of 1/scale (the half storage format)
// and `is` = 1/scale: every term is linear in (f, F) except rho = 1 + drho,
// rho vv and vF + Fv, which take one factor `is` each; the outputs come out
// in the same scaled units.
// With VOUT the fluid velocity v = (j + F/2) / rho of Eq. (macrovariables2)
// is also returned in v3, in physical units (the same expression, rounding
// for rounding, as macro19).
// `out` is an array of NQ, or (packed path) a callable out(i, value) that
// consumes each population as soon as it is known, so that the stores of
// the first ones are issued before the last are computed.
template <typename O, typename T>
__device__ __forceinline__ void put(O& out, int i, T v) {
    if constexpr (std::is_pointer<O>::value)
        out[i] = v;
    else
        out(i, v);
}
template <typename T, bool COMP, bool SCALED = false, bool VOUT = false, typename O>
__device__ __forceinline__ void collide19(const T f[NQ], T Fx, T Fy, T Fz, const Coef<T>& k, O out,
                                          T is = T(1), T* v3 = nullptr) {
    using W = Wts<T>;
    constexpr bool PACKED = std::is_same<T, F2>::value;
    // FP64 keeps 53 bits against the tolerance's 40, so it takes the same
    // folded reconstruction as the 16-bit formats (fewer FP64 operations,
    // each an issue of the SM's FP64 unit); FP32 keeps the ordering that
    // rounds the momentum term once.
    constexpr bool FOLD = PACKED || std::is_same<T, double>::value;
    const Moments<T> m = moments19<T, COMP>(f);
    const T third = T(1) / T(3);
    const T rho = T(1) + (SCALED ? m.drho * is : m.drho);
    T irho;
    if constexpr (PACKED) {  // the 16-bit formats: an approximate reciprocal, 2 ulp of float
        irho = F2(make_float2(__fdividef(1.0f, rho.v.x), __fdividef(1.0f, rho.v.y)));
    } else if constexpr (std::is_same<T, double>::value) {
        // Newton-Raphson from the float reciprocal (relative error e ->
        // e^2 per step: 2^-23 -> 2^-46 -> about one unit in the last
        // place), four FP64 operations in place of a division
        double r = (double)__frcp_rn((float)rho);
        r = r * fma(-rho, r, 2.0);
        irho = r * fma(-rho, r, 2.0);
    } else {
        irho = T(1) / rho;
    }
    if (VOUT) {
        const T iv = SCALED ? is * irho : irho;
        v3[0] = (m.jx + (COMP ? m.jx_lo + T(0.5) * Fx : T(0.5) * Fx)) * iv;
        v3[1] = (m.jy + (COMP ? m.jy_lo + T(0.5) * Fy : T(0.5) * Fy)) * iv;
        v3[2] = (m.jz + (COMP ? m.jz_lo + T(0.5) * Fz : T(0.5) * Fz)) * iv;
    }
    const T vx = (m.jx + T(0.5) * Fx) * irho;
    const T vy = (m.jy + T(0.5) * Fy) * irho;
    const T vz = (m.jz + T(0.5) * Fz) * irho;
    const T rs = SCALED ? rho * is : rho;
    const T Fxs = SCALED ? Fx * is : Fx, Fys = SCALED ? Fy * is : Fy, Fzs = SCALED ? Fz * is : Fz;
    // S = P - (drho/3) 1 ; X = S - rho vv ; Y = vF + Fv
    const T sxx = m.pxx - third * m.drho, syy = m.pyy - third * m.drho, szz = m.pzz - third * m.drho;
    const T xxx = sxx - rs * vx * vx, xyy = syy - rs * vy * vy, xzz = szz - rs * vz * vz;
    const T xxy = m.pxy - rs * vx * vy, xxz = m.pxz - rs * vx * vz, xyz = m.pyz - rs * vy * vz;
    const T yxx = T(2) * vx * Fxs, yyy = T(2) * vy * Fys, yzz = T(2) * vz * Fzs;
    const T yxy = vx * Fys + Fxs * vy, yxz = vx * Fzs + Fxs * vz, yyz = vy * Fzs + Fys * vz;
    const T trX = xxx + xyy + xzz, trY = yxx + yyy + yzz;
    const T dev_tr = third * (trX - k.tau_s * trY);
    const T iso = third * k.om_b * (trX - k.tau_b * trY);
    const T bxx = sxx - k.om_s * (xxx - k.tau_s * yxx - dev_tr) - iso;
    const T byy = syy - k.om_s * (xyy - k.tau_s * yyy - dev_tr) - iso;
    const T bzz = szz - k.om_s * (xzz - k.tau_s * yzz - dev_tr) - iso;
    const T bxy = m.pxy - k.om_s * (xxy - k.tau_s * yxy);
    const T bxz = m.pxz - k.om_s * (xxz - k.tau_s * yxz);
    const T byz = m.pyz - k.om_s * (xyz - k.tau_s * yyz);

    const T base = m.drho - T(1.5) * (bxx + byy + bzz);
    put(out, 0, W::w0 * base);
    // axis populations: w1 (base + 4.5 B_aa) + a1 (+-F_a) + a1 (+-j_a)
    const T hx = W::w1 * (base + T(4.5) * bxx), hy = W::w1 * (base + T(4.5) * byy),
            hz = W::w1 * (base + T(4.5) * bzz);
    // force density plus the low part of j: both are far smaller than j
    const T Gx = COMP ? Fx + m.jx_lo : Fx, Gy = COMP ? Fy + m.jy_lo : Fy, Gz = COMP ? Fz + m.jz_lo : Fz;
    if constexpr (FOLD) {
        // The 16-bit formats round their storage at 2^-11 (half) or 2^-8
        // (bfloat16) relative, far above the rounding of A = j + F in
        // float, and FP64 far below its tolerance, so the force is folded
        // into j first and each population pair (c, -c) shares its odd
        // part: out = even +- w A.c / c_s^2.
        const T Ax = m.jx + Gx, Ay = m.jy + Gy, Az = m.jz + Gz;
        const T ox = W::a1 * Ax, oy = W::a1 * Ay, oz = W::a1 * Az;
        put(out, 1, hx + ox);
        put(out, 2, hx - ox);
        put(out, 3, hy + oy);
        put(out, 4, hy - oy);
        put(out, 5, hz + oz);
        put(out, 6, hz - oz);
        // face diagonals in plane (a, b), populations n..n+3 with
        // c = (+,+), (-,-), (+,-), (-,+)
        const auto plane = [&](int n, T baa_bb, T bab, T Aa, T Ab) {
            const T p = base + T(4.5) * baa_bb, q = T(9) * bab;
            const T gp = W::w2 * (p + q), gm = W::w2 * (p - q);
            const T op = W::b1 * (Aa + Ab), om = W::b1 * (Aa - Ab);
            put(out, n, gp + op);
            put(out, n + 1, gp - op);
            put(out, n + 2, gm + om);
            put(out, n + 3, gm - om);
        };
        plane(7, bxx + byy, bxy, Ax, Ay);
        plane(11, bxx + bzz, bxz, Ax, Az);
        plane(15, byy + bzz, byz, Ay, Az);
        return;
    }
    const T pxy_ = base + T(4.5) * (bxx + byy), pxz_ = base + T(4.5) * (bxx + bzz), pyz_ = base + T(4.5) * (byy + bzz);
    const T qxy = T(9) * bxy, qxz = T(9) * bxz, qyz = T(9) * byz;
    const T gpxy = W::w2 * (pxy_ + qxy), gmxy = W::w2 * (pxy_ - qxy);
    const T gpxz = W::w2 * (pxz_ + qxz), gmxz = W::w2 * (pxz_ - qxz);
    const T gpyz = W::w2 * (pyz_ + qyz), gmyz = W::w2 * (pyz_ - qyz);
    const T fx = W::a1 * Gx, fy = W::a1 * Gy, fz = W::a1 * Gz;
    put(out, 1, fma(W::a1, m.jx, hx + fx));
    put(out, 2, fma(-W::a1, m.jx, hx - fx));
    put(out, 3, fma(W::a1, m.jy, hy + fy));
    put(out, 4, fma(-W::a1, m.jy, hy - fy));
    put(out, 5, fma(W::a1, m.jz, hz + fz));
    put(out, 6, fma(-W::a1, m.jz, hz - fz));
    // face diagonals (s1, s2) in plane (a, b):
    //   w2 (base + 4.5 (B_aa + B_bb) + 9 s1 s2 B_ab) + b1 (s1 F_a + s2 F_b) + b1 (s1 j_a + s2 j_b)
    const T Fpxy = W::b1 * (Gx + Gy), Fmxy = W::b1 * (Gx - Gy);
    const T Fpxz = W::b1 * (Gx + Gz), Fmxz = W::b1 * (Gx - Gz);
    const T Fpyz = W::b1 * (Gy + Gz), Fmyz = W::b1 * (Gy - Gz);
    const T b = W::b1;
    put(out, 7, fma(b, m.jx, fma(b, m.jy, gpxy + Fpxy)));
    put(out, 8, fma(-b, m.jx, fma(-b, m.jy, gpxy - Fpxy)));
    put(out, 9, fma(b, m.jx, fma(-b, m.jy, gmxy + Fmxy)));
    put(out, 10, fma(-b, m.jx, fma(b, m.jy, gmxy - Fmxy)));
    put(out, 11, fma(b, m.jx, fma(b, m.jz, gpxz + Fpxz)));
    put(out, 12, fma(-b, m.jx, fma(-b, m.jz, gpxz - Fpxz)));
    put(out, 13, fma(b, m.jx, fma(-b, m.jz, gmxz + Fmxz)));
    put(out, 14, fma(-b, m.jx, fma(b, m.jz, gmxz - Fmxz)));
    put(out, 15, fma(b, m.jy, fma(b, m.jz, gpyz + Fpyz)));
    put(out, 16, fma(-b, m.jy, fma(-b, m.jz, gpyz - Fpyz)));
    put(out, 17, fma(b, m.jy, fma(-b, m.jz, gmyz + Fmyz)));
    put(out, 18, fma(-b, m.jy, fma(b, m.jz, gmyz - Fmyz)));
}

// drho = rho - 1 and v = (j + F/2) / rho, Eq. (macrovariables2).
template <typename T, bool COMP = false>
__device__ __forceinline__ void macro19(const T f[NQ], T Fx, T Fy, T Fz, T& drho, T& vx, T& vy, T& vz) {
    const Moments<T> m = moments19<T, COMP>(f);
    drho = m.drho;
    const T rho = T(1) + m.drho;
    const T irho = T(1) / rho;
    vx = (m.jx + (m.jx_lo + T(0.5) * Fx)) * irho;
    vy = (m.jy + (m.jy_lo + T(0.5) * Fy)) * irho;
    vz = (m.jz + (m.jz_lo + T(0.5) * Fz)) * irho;
}

// ------------------------------------------------------- Peskin kernel
// phi(r) of Sec. III, Eq. (deltadef): support |r| < 2.
__device__ __forceinline__ double peskin_phi(double r) {
    const double s = fabs(r);
    if (s <= 1.0) return (3.0 - 2.0 * s + sqrt(1.0 + 4.0 * s - 4.0 * s * s)) * 0.125;
    if (s <= 2.0) return (5.0 - 2.0 * s - sqrt(-7.0 + 12.0 * s - 4.0 * s * s)) * 0.125;
    return 0.0;
}
__device__ __forceinline__ float peskin_phi(float r) {
    const float s = fabsf(r);
    if (s <= 1.0f) return (3.0f - 2.0f * s + sqrtf(1.0f + 4.0f * s - 4.0f * s * s)) * 0.125f;
    if (s <= 2.0f) return (5.0f - 2.0f * s - sqrtf(-7.0f + 12.0f * s - 4.0f * s * s)) * 0.125f;
    return 0.0f;
}

// Stencil of one axis for a position X in [0, n): nodes floor(X)-1 ..
// floor(X)+2; node k's offset from X is (floor(X) - 1 + k) - X.
__device__ __forceinline__ int stencil_base(double X) { return (int)floor(X) - 1; }
__device__ __forceinline__ int wrap_node(int k, int n) {
    // k in [-1, n + 2): one correction suffices for n >= 3; the modulo
    // covers the smaller lattices, where a stencil may wrap twice
    if (n >= 3) return k < 0 ? k + n : (k >= n ? k - n : k);
    int r = k % n;
    return r < 0 ? r + n : r;
}

// The 4 x 4 x 4 stencil of one point, evaluated by a warp: lane 4a + i
// (lanes 0-11) holds the base node of axis a and the one-dimensional weight
// phi(b_a + i - X_a) of Eq. (deltadef), from FP64 position arithmetic; every
// lane reads the weights of its nodes by shuffle, so the 64 nodes cost 12
// evaluations of phi.  The weight of node (i, j, k) is
// (phi_x[i] phi_y[j]) phi_z[k].
template <typename T>
struct StencilLane {
    T phi;
    int base;
};
template <typename T>
__device__ __forceinline__ StencilLane<T> stencil_lane(double X, double Y, double Z, int lane) {
    StencilLane<T> s;
    s.phi = T(0);
    s.base = 0;
    if (lane < 12) {
        const int a = lane >> 2, i = lane & 3;
        const double P = a == 0 ? X : (a == 1 ? Y : Z);
        s.base = stencil_base(P);
        s.phi = peskin_phi((T)((double)(s.base + i) - P));
    }
    return s;
}

// Stencil row of a point, computed once per position by a thread per point
// and read by the warp-per-point kernels: elements 0-11 hold phi(b_a + i -
// X_a) (axis a, node i at 4a + i), elements 12-14 the base nodes b_a as int
// bits, element 15 is unused; 16 elements of the arithmetic type, so a
// warp reads a row with one coalesced load.
constexpr int ST_W = 16;
__device__ __forceinline__ float int_bits(int v, float) { return __int_as_float(v); }
__device__ __forceinline__ double int_bits(int v, double) { return __longlong_as_double((long long)v); }
__device__ __forceinline__ int bits_int(float v) { return __float_as_int(v); }
__device__ __forceinline__ int bits_int(double v) { return (int)__double_as_longlong(v); }

template <typename T>
__device__ __forceinline__ void write_stencil(T* __restrict__ row, double X, double Y, double Z) {
    const double P[3] = {X, Y, Z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int b = stencil_base(P[a]);
#pragma unroll
        for (int i = 0; i < 4; ++i) row[4 * a + i] = peskin_phi((T)((double)(b + i) - P[a]));
        row[12 + a] = int_bits(b, T(0));
    }
    row[15] = T(0);
}

}  // namespace lbk
