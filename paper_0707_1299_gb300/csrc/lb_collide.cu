// lb_collide.cu -- the collide+stream kernels (Sec. II, Eq. fiexp with the
// stress update of Eq. mrtlbe) and their launcher:
//   k_collide       one thread per site, all storage formats;
//   k_collide_pair  the 16-bit formats with nx even: two sites a thread,
//                   packed FP32x2 arithmetic;
//   k_fixup         recomputes the few force tiles of fixed points after a
//                   field-free collide.
// Kept apart from the other kernels so that a change elsewhere does not
// invalidate the committed ncu traffic figure of k_collide.
#include <math.h>

#include <algorithm>

#include "../../include/lb.h"
#include "lb_internal.h"

namespace lbk {

// Collision and store of one site from its pulled populations f: force =
// uniform + (field ? localised : 0), in the stored units of the format;
// with VOUT and a field, v = (j + F/2) / rho is written to vel as well and
// the consumed force is zeroed (VOUT is the mode of mobile colloids, whose
// field is spread anew every step).
template <typename S, bool VOUT>
__device__ __forceinline__ void finish_site(const typename Store<S>::T (&f)[NQ], const Pops<S>& dst,
                                            typename Store<S>::T* floc,
                                            typename Store<S>::T* __restrict__ vel, unsigned site,
                                            bool field, const Coef<typename Store<S>::T>& k,
                                            const UForce<typename Store<S>::T>& fu, float scale, float inv_scale,
                                            unsigned seed) {
    using T = typename Store<S>::T;
    constexpr bool SC = Store<S>::kScaled;
    T Fx = fu.F[0], Fy = fu.F[1], Fz = fu.F[2];
    if (field) {  // read-only path: see reset_group_flag
        const T s = SC ? (T)scale : T(1);
        T lx, ly, lz;
        field_ldg(floc, site, lx, ly, lz);
        Fx += lx * s;
        Fy += ly * s;
        Fz += lz * s;
    }
    T o[NQ], v3[3];
    collide19<T, Store<S>::kCompensate, SC, VOUT>(f, Fx, Fy, Fz, k, o, (T)inv_scale, v3);
    unsigned rn = rng_seed(site, seed);
#pragma unroll
    for (int i = 0; i < NQ; ++i) Store<S>::st(dst.p[i], site, o[i], rng_next(rn));
    if (VOUT && field) {
        field_st(vel, site, v3[0], v3[1], v3[2]);
        field_st(floc, site, T(0), T(0), T(0));  // the consumed force
    }
}

// With VOUT, the first lane of each flagged 8-site group resets the group's
// flag once the group's sites are done.  The flag word and the field are
// read through the read-only (non-coherent) path although this kernel
// writes them afterwards: each flag word is read by one warp-wide load of
// the one warp that owns its tile, and each field value by the one thread
// of its site, always before that warp or thread overwrites it; nothing
// else reads them in the launch.  (Coherent loads of the two measured 9 %
// slower on the FP32 colloid step at 512^3 on GB300.)
__device__ __forceinline__ void reset_group_flag(flag_t* flags, unsigned tile, unsigned x_in_tile, unsigned fl) {
    if (fl && x_in_tile % GROUP_X == 0) flags[tile * (TILE_X / GROUP_X) + x_in_tile / GROUP_X] = 0;
}

// With VOUT, a warp also asks L2 for the force lines of the flagged groups
// of its tile row in the next plane, whose collide follows about a plane's
// worth of blocks later: that warp then finds its dependent force loads in
// L2.  One extra flag word a warp and a prefetch per flagged group; at 512^3
// with 1e5 colloids the FP32 collide took 3.216 against 3.241 ms (two planes
// ahead 3.227, three 3.261).
template <typename T>
__device__ __forceinline__ void prefetch_next_forces(const T* floc, const flag_t* flags, const Geom& g, int z, int y,
                                                     unsigned tx, unsigned x, unsigned x_in_tile) {
    const int zq = (z + 1) % g.nz;
    const unsigned tq = ((unsigned)zq * (unsigned)g.ny + (unsigned)y) * (unsigned)g.ntx + tx;
    const unsigned wq = __ldg((const unsigned*)flags + tq);
    if (group_flag(wq, x_in_tile) && x_in_tile % GROUP_X == 0) {
        const size_t sq = (size_t)zq * g.plane + (size_t)y * (size_t)g.nx + x;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(floc + FIELD_W * sq));
    }
}

// ------------------------------------------------------------ k_collide
// NY consecutive y rows per thread (all loads of the NY sites issued
// first).  The half format is handled in its scaled units throughout.
// Occupancy bound (blocks of 128 threads per SM), swept on GB300 at 256^3:
// the 4- and 2-byte formats are fastest at 12 (42 registers; 8-10 were
// 2-10 % slower, 14 spills); FP64 at 8.
// FMODE: FM_NONE a lattice without point forces (no flag or field access);
// FM_FIELD the force field is read in flagged groups; FM_VEL also writes the
// fluid velocity v = (j + F/2) / rho there, for the colloid update, and
// zeroes the consumed field and flags (so no clearing pass follows).
enum { FM_NONE = 0, FM_FIELD = 1, FM_VEL = 2 };
template <typename S, bool WALLS, int NY, int FMODE>
__global__ void __launch_bounds__(CS_THREADS, (NY == 1 ? (sizeof(S) == 8 ? 8 : 12) : 4))
k_collide(const Pops<S> src, const Pops<S> dst, typename Store<S>::T* __restrict__ floc,
          flag_t* __restrict__ flags, typename Store<S>::T* __restrict__ vel, Geom g,
          Coef<typename Store<S>::T> k, UForce<typename Store<S>::T> fu, float scale, float inv_scale,
          unsigned seed) {
    using T = typename Store<S>::T;
    constexpr bool FIELD = FMODE != FM_NONE, VOUT = FMODE == FM_VEL;
    const int y0 = (blockIdx.y * CS_WARPS + threadIdx.y) * NY;
    if (y0 >= g.ny) return;  // uniform per warp
    const int z = blockIdx.z, lane = threadIdx.x;
    const int x = blockIdx.x * TILE_X + lane;
    unsigned fl[NY];
#pragma unroll
    for (int r = 0; r < NY; ++r) {
        const unsigned tile = ((unsigned)z * (unsigned)g.ny + (unsigned)(y0 + r)) * (unsigned)g.ntx + blockIdx.x;
        fl[r] = (FIELD && y0 + r < g.ny) ? group_flag(__ldg((const unsigned*)flags + tile), lane) : 0u;
    }

    if (x < g.nx) {
        if (WALLS && is_solid(g, z)) {
#pragma unroll
            for (int r = 0; r < NY; ++r) {
                if (y0 + r >= g.ny) break;
                const unsigned site = (unsigned)z * g.plane + (unsigned)(y0 + r) * (unsigned)g.nx + (unsigned)x;
#pragma unroll
                for (int i = 0; i < NQ; ++i) Store<S>::st(dst.p[i], site, T(0), 0u);
            }
        } else {
            T f[NY][NQ];
            Nbr n[NY];
#pragma unroll
            for (int r = 0; r < NY; ++r)  // every load of the NY sites first
                if (y0 + r < g.ny) {
                    n[r] = neighbours(g, x, y0 + r, z);
                    pull19<S, WALLS>(src, n[r], f[r]);
                }
            if (VOUT) prefetch_next_forces(floc, flags, g, z, y0, blockIdx.x, (unsigned)x, (unsigned)lane);
#pragma unroll
            for (int r = 0; r < NY; ++r) {
                if (y0 + r >= g.ny) break;
                // the field loads come after the population loads, so both are in flight together
                finish_site<S, VOUT>(f[r], dst, floc, vel, n[r].c + n[r].x, FIELD && fl[r], k, fu, scale, inv_scale,
                                     seed);
            }
        }
    }
    if (VOUT)
#pragma unroll
        for (int r = 0; r < NY; ++r)
            if (y0 + r < g.ny)
                reset_group_flag(flags, ((unsigned)z * (unsigned)g.ny + (unsigned)(y0 + r)) * (unsigned)g.ntx + blockIdx.x,
                                 (unsigned)lane, fl[r]);
}

// The collide for the 16-bit formats with nx even: two x-adjacent sites
// per thread, one 32-bit word per population and site pair, and the two
// sites' arithmetic on the packed FP32x2 datapath (F2), so a site costs
// half the load, store and floating-point instructions of k_collide (the
// instruction count, not the bytes, bounds these formats).  Each word is
// rounded by one stochastic-rounding conversion of the pair, from one
// random draw of a stream seeded by the pair's first site; the arithmetic
// differs from k_collide's in its reciprocal of rho and in folding F into
// j before the odd parts (see collide19).
// Grid: (ceil(nx / 64), ceil(ny / 4), nz).  Occupancy bound (blocks of 128
// threads per SM) and store order, swept on GB300 at 256^3 (the four
// lattices of the channel workload): half 8 blocks (64 registers) with the
// stores after the arithmetic; bfloat16 9 blocks (56 registers) with each
// store issued as its population is known.  The other combinations, and 6,
// 7 or 10 blocks, were 1-6 % slower.
template <typename S, bool WALLS, int FMODE>
__global__ void __launch_bounds__(CS_THREADS, Store<S>::kScaled ? 8 : 9)
k_collide_pair(const Pops<S> src, const Pops<S> dst, float* __restrict__ floc, flag_t* __restrict__ flags,
               float* __restrict__ vel, Geom g, Coef<float> k, UForce<float> fu, float scale, float inv_scale,
               unsigned seed) {
    using St = Store<S>;
    constexpr bool SC = St::kScaled, FIELD = FMODE != FM_NONE, VOUT = FMODE == FM_VEL;
    const int y = blockIdx.y * CS_WARPS + threadIdx.y;
    if (y >= g.ny) return;  // uniform per warp
    const int z = blockIdx.z, lane = threadIdx.x;
    const unsigned nx = (unsigned)g.nx;
    const unsigned x0 = (blockIdx.x * 32u + (unsigned)lane) * 2u;
    const bool active = x0 < nx;
    const unsigned row = (unsigned)z * g.plane + (unsigned)y * nx;
    if (WALLS && is_solid(g, z)) {  // uniform per warp
        if (active)
#pragma unroll
            for (int i = 0; i < NQ; ++i) *(unsigned*)(dst.p[i] + row + x0) = 0u;
        return;
    }
    const unsigned tile = ((unsigned)z * (unsigned)g.ny + (unsigned)y) * (unsigned)g.ntx + x0 / TILE_X;
    const unsigned fl = (FIELD && active) ? group_flag(__ldg((const unsigned*)flags + tile), x0 % TILE_X) : 0u;
    const Nbr n = neighbours(g, 0, y, z);
    unsigned w[NQ];
    float4 fs0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), fs1 = fs0;  // the two sites' force words
    // the force loads are issued after the population loads and before the
    // shuffles wait for those, so both are in flight together
    pull19_pair<S, WALLS>(src, n, x0, nx, lane, active, w, [&] {
        if (FIELD && fl) {
            fs0 = __ldg((const float4*)floc + row + x0);
            fs1 = __ldg((const float4*)floc + row + x0 + 1);
        }
    });
    const float2 fa = make_float2(fs0.x, fs1.x), fb = make_float2(fs0.y, fs1.y), fc = make_float2(fs0.z, fs1.z);
    F2 f[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) f[i] = F2(St::unpack2(w[i]));
    F2 Fx(fu.F[0]), Fy(fu.F[1]), Fz(fu.F[2]);
    if (FIELD && fl) {
        const F2 sc(SC ? scale : 1.0f);
        Fx = fma(F2(fa), sc, Fx);
        Fy = fma(F2(fb), sc, Fy);
        Fz = fma(F2(fc), sc, Fz);
    }
    Coef<F2> k2;
    k2.tau_s = F2(k.tau_s);
    k2.tau_b = F2(k.tau_b);
    k2.om_s = F2(k.om_s);
    k2.om_b = F2(k.om_b);
    F2 v3[3];
    unsigned rs = rng_seed(row + x0, seed);
    if constexpr (SC) {  // half: all populations first, then the stores
        F2 o[NQ];
        collide19<F2, false, SC, VOUT>(f, Fx, Fy, Fz, k2, o, F2(inv_scale), v3);
        if (active)
#pragma unroll
            for (int i = 0; i < NQ; ++i)
                *(unsigned*)(dst.p[i] + row + x0) = St::bits2_rs(o[i].v.x, o[i].v.y, rng_next2(rs));
    } else {  // bfloat16: each population is rounded and stored as soon as it is computed
        const auto emit = [&](int i, F2 v) {
            const unsigned word = St::bits2_rs(v.v.x, v.v.y, rng_next2(rs));
            if (active) *(unsigned*)(dst.p[i] + row + x0) = word;
        };
        collide19<F2, false, SC, VOUT>(f, Fx, Fy, Fz, k2, emit, F2(inv_scale), v3);
    }
    if (VOUT && fl && active) {
        field_st(vel, row + x0, v3[0].v.x, v3[1].v.x, v3[2].v.x);
        field_st(vel, row + x0 + 1, v3[0].v.y, v3[1].v.y, v3[2].v.y);
        field_st(floc, row + x0, 0.0f, 0.0f, 0.0f);  // the consumed force
        field_st(floc, row + x0 + 1, 0.0f, 0.0f, 0.0f);
    }
    if (VOUT) reset_group_flag(flags, tile, x0 % TILE_X, fl);
}

// The collide for the 16-bit formats with nx a multiple of 4: four
// x-adjacent sites a thread, one 64-bit word per population loaded
// (pull19_quad), so a site costs half the load instructions of
// k_collide_pair and each load moves twice the bytes (the pair kernel is
// bound by memory latency at its occupancy: more bytes in flight a warp).
// The two site pairs run one after the other through the packed FP32x2
// collision of k_collide_pair, each rounded to a 32-bit word by the
// stochastic-rounding conversion (one random stream a thread, seeded by its
// first site), and the two words of a population go out as one 64-bit store.
// The four sites share one 8-site force group.  Occupancy bound, measured on
// GB300: 5 blocks an SM without a force field (96 registers), 4 with one
// (where 5 spills): 512^3 with 1e5 colloids, half storage, 1.887 ms against
// 1.936 at 5; field-free 256^3, 0.214 ms against 0.232 at 4.
// Grid: (ceil(nx / 128), ceil(ny / 4), nz).
template <typename S, bool WALLS, int FMODE>
__global__ void __launch_bounds__(CS_THREADS, FMODE == FM_NONE ? 5 : 4)
k_collide_quad(const Pops<S> src, const Pops<S> dst, float* __restrict__ floc, flag_t* __restrict__ flags,
               float* __restrict__ vel, Geom g, Coef<float> k, UForce<float> fu, float scale, float inv_scale,
               unsigned seed) {
    using St = Store<S>;
    constexpr bool SC = St::kScaled, FIELD = FMODE != FM_NONE, VOUT = FMODE == FM_VEL;
    const int y = blockIdx.y * CS_WARPS + threadIdx.y;
    if (y >= g.ny) return;  // uniform per warp
    const int z = blockIdx.z, lane = threadIdx.x;
    const unsigned nx = (unsigned)g.nx;
    const unsigned x0 = (blockIdx.x * 32u + (unsigned)lane) * 4u;
    const bool active = x0 < nx;
    const unsigned row = (unsigned)z * g.plane + (unsigned)y * nx;
    if (WALLS && is_solid(g, z)) {  // uniform per warp
        if (active)
#pragma unroll
            for (int i = 0; i < NQ; ++i) *(uint2*)(dst.p[i] + row + x0) = make_uint2(0u, 0u);
        return;
    }
    const unsigned tile = ((unsigned)z * (unsigned)g.ny + (unsigned)y) * (unsigned)g.ntx + x0 / TILE_X;
    const unsigned fl = (FIELD && active) ? group_flag(__ldg((const unsigned*)flags + tile), x0 % TILE_X) : 0u;
    const Nbr n = neighbours(g, 0, y, z);
    unsigned lo[NQ], hi[NQ];
    float4 fs[4];  // the four sites' force words
#pragma unroll
    for (int q = 0; q < 4; ++q) fs[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    pull19_quad<S, WALLS>(src, n, x0, nx, lane, active, lo, hi, [&] {
        if (FIELD && fl)  // in flight with the population loads
#pragma unroll
            for (int q = 0; q < 4; ++q) fs[q] = __ldg((const float4*)floc + row + x0 + q);
    });
    F2 Fx[2] = {F2(fu.F[0]), F2(fu.F[0])}, Fy[2] = {F2(fu.F[1]), F2(fu.F[1])}, Fz[2] = {F2(fu.F[2]), F2(fu.F[2])};
    if (FIELD && fl) {
        const float sc = SC ? scale : 1.0f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            Fx[h] = fma(F2(make_float2(fs[2 * h].x, fs[2 * h + 1].x)), F2(sc), Fx[h]);
            Fy[h] = fma(F2(make_float2(fs[2 * h].y, fs[2 * h + 1].y)), F2(sc), Fy[h]);
            Fz[h] = fma(F2(make_float2(fs[2 * h].z, fs[2 * h + 1].z)), F2(sc), Fz[h]);
        }
    }
    Coef<F2> k2;
    k2.tau_s = F2(k.tau_s);
    k2.tau_b = F2(k.tau_b);
    k2.om_s = F2(k.om_s);
    k2.om_b = F2(k.om_b);
    F2 v3[2][3];
    unsigned rs = rng_seed(row + x0, seed);
    unsigned keep[NQ];  // the first pair's rounded words, stored with the second's
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // the site pairs (x0, x0 + 1) and (x0 + 2, x0 + 3)
        F2 f[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) f[i] = F2(St::unpack2(h ? hi[i] : lo[i]));
        // each population of the second pair is rounded and stored, with
        // the first pair's word, as soon as it is computed: one 64-bit store
        // a population (a warp writes 256 contiguous bytes), not two 32-bit
        // ones that each fill half of every sector they touch
        const auto emit = [&](int i, F2 v) {
            const unsigned word = St::bits2_rs(v.v.x, v.v.y, rng_next2(rs));
            if (h == 0) keep[i] = word;
            else if (active) *(uint2*)(dst.p[i] + row + x0) = make_uint2(keep[i], word);
        };
        collide19<F2, false, SC, VOUT>(f, Fx[h], Fy[h], Fz[h], k2, emit, F2(inv_scale), v3[h]);
    }
    if (VOUT && fl && active) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            field_st(vel, row + x0 + 2 * h, v3[h][0].v.x, v3[h][1].v.x, v3[h][2].v.x);
            field_st(vel, row + x0 + 2 * h + 1, v3[h][0].v.y, v3[h][1].v.y, v3[h][2].v.y);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) field_st(floc, row + x0 + q, 0.0f, 0.0f, 0.0f);  // the consumed force
    }
    if (VOUT) reset_group_flag(flags, tile, x0 % TILE_X, fl);
}

// Fix-up for a few fixed points: the collide ran with the uniform force at
// every site (FM_NONE); one warp per listed tile recomputes its sites with
// the localised force added and overwrites them, with the same arithmetic
// and the same rounding bits as the field-aware collide.  Solid sites carry
// no force (the spread skips them), so they are left as they are.
template <typename S, bool WALLS>
__global__ void __launch_bounds__(CS_THREADS)
k_fixup(const Pops<S> src, const Pops<S> dst, typename Store<S>::T* __restrict__ floc,
        const unsigned* __restrict__ list, const unsigned* __restrict__ count, Geom g, Coef<typename Store<S>::T> k,
        UForce<typename Store<S>::T> fu, float scale, float inv_scale, unsigned seed) {
    using T = typename Store<S>::T;
    const unsigned w = blockIdx.x * CS_WARPS + threadIdx.y;
    if (w >= __ldg(count)) return;
    const unsigned tile = list[w];
    const unsigned row = tile / (unsigned)g.ntx;
    const int x = (int)(tile - row * (unsigned)g.ntx) * TILE_X + threadIdx.x;
    const int y = (int)(row % (unsigned)g.ny), z = (int)(row / (unsigned)g.ny);
    if (x >= g.nx || (WALLS && is_solid(g, z))) return;
    const Nbr n = neighbours(g, x, y, z);
    T f[NQ];
    pull19<S, WALLS>(src, n, f);
    finish_site<S, false>(f, dst, floc, nullptr, n.c + n.x, true, k, fu, scale, inv_scale, seed);
}

// The pair kernel exists for the 16-bit formats; for the others PairS maps
// to a 16-bit type only to keep the dead branch of LB_COLLIDE compilable.
template <typename S> struct PairSel { using type = __half; };
template <> struct PairSel<__nv_bfloat16> { using type = __nv_bfloat16; };
template <typename S> using PairS = typename PairSel<S>::type;
template <typename T> static Coef<float> coef_f(const Coef<T>& k) {
    Coef<float> r;
    r.tau_s = (float)k.tau_s;
    r.tau_b = (float)k.tau_b;
    r.om_s = (float)k.om_s;
    r.om_b = (float)k.om_b;
    return r;
}
template <typename T> static UForce<float> uforce_f(const UForce<T>& u) {
    UForce<float> r;
    for (int a = 0; a < 3; ++a) r.F[a] = (float)u.F[a];
    return r;
}

template <typename S>
static cudaError_t collide_t(lb_ctx* c) {
    using T = typename Store<S>::T;
    Coef<T> k;
    k.tau_s = (T)c->tau_s;
    k.tau_b = (T)c->tau_b;
    k.om_s = (T)(1.0 / (c->tau_s + 0.5));
    k.om_b = (T)(1.0 / (c->tau_b + 0.5));
    const Pops<S> src = pops<S>(c->f[c->cur], c->geom.V), dst = pops<S>(c->f[1 - c->cur], c->geom.V);
    UForce<T> fu = uniform_force<T>(c);
    if (Store<S>::kScaled)
        for (int a = 0; a < 3; ++a) fu.F[a] = (T)((double)fu.F[a] * (double)c->scale);
    // one site per thread for every format: two rows per thread (more loads
    // in flight for the 2-byte formats) measured slower on GB300 (fewer
    // resident warps at 80-92 registers)
    constexpr int NY = 1;
    const dim3 grid((unsigned)c->geom.ntx, (unsigned)((c->geom.ny + CS_WARPS * NY - 1) / (CS_WARPS * NY)),
                    (unsigned)c->geom.nz);
    T* floc = (T*)c->floc;
    T* vel = (T*)c->vel;
    // a few fixed points: field-free collide plus the fix-up of their tiles
    const bool fixup = c->npts > 0 && c->n_mobile == 0 && c->fix_ok;
    const int mode = (c->npts == 0 || fixup) ? FM_NONE : (c->n_mobile > 0 ? FM_VEL : FM_FIELD);
    // the 16-bit formats take two sites a thread when the rows pair up
    constexpr bool PAIRABLE = sizeof(S) == 2;
    const bool pair = PAIRABLE && (c->geom.nx % 2) == 0;
    // four sites a thread (64-bit loads and stores) wherever the rows allow:
    // at 512^3 with 1e5 colloids, 1.99 (half) and 2.01 ms (bfloat16) a step
    // against 2.26 and 2.19 ms with the pair kernel
    const bool quad = PAIRABLE && (c->geom.nx % 4) == 0;
    const dim3 pgrid((unsigned)((c->geom.nx + 63) / 64), grid.y, grid.z);
    const dim3 qgrid((unsigned)((c->geom.nx + 127) / 128), grid.y, grid.z);
#define LB_COLLIDE(W, FM)                                                                                          \
    do {                                                                                                           \
        if (PAIRABLE && quad)                                                                                      \
            k_collide_quad<PairS<S>, W, FM><<<qgrid, site_block(), 0, c->stream>>>(                                \
                pops<PairS<S>>(c->f[c->cur], c->geom.V), pops<PairS<S>>(c->f[1 - c->cur], c->geom.V),              \
                (float*)floc, c->flags, (float*)vel, c->geom, coef_f(k), uforce_f(fu), c->scale, c->inv_scale, \
                c->seed);                                                                                          \
        else if (PAIRABLE && pair)                                                                                 \
            k_collide_pair<PairS<S>, W, FM><<<pgrid, site_block(), 0, c->stream>>>(                                \
                pops<PairS<S>>(c->f[c->cur], c->geom.V), pops<PairS<S>>(c->f[1 - c->cur], c->geom.V),              \
                (float*)floc, c->flags, (float*)vel, c->geom, coef_f(k), uforce_f(fu), c->scale, c->inv_scale, \
                c->seed);                                                                                          \
        else                                                                                                       \
            k_collide<S, W, NY, FM><<<grid, site_block(), 0, c->stream>>>(src, dst, floc, c->flags, vel, c->geom,  \
                                                                        k, fu, c->scale, c->inv_scale, c->seed);   \
    } while (0)
    if (has_walls(c)) {
        if (mode == FM_VEL) LB_COLLIDE(true, FM_VEL);
        else if (mode == FM_FIELD) LB_COLLIDE(true, FM_FIELD);
        else LB_COLLIDE(true, FM_NONE);
    } else {
        if (mode == FM_VEL) LB_COLLIDE(false, FM_VEL);
        else if (mode == FM_FIELD) LB_COLLIDE(false, FM_FIELD);
        else LB_COLLIDE(false, FM_NONE);
    }
#undef LB_COLLIDE
    c->launches++;
    if (fixup) {  // one warp per listed tile; the count is read on the device
        const unsigned cap = fixed_tile_cap(c);
        const unsigned* count = c->fix_list + cap;
        const unsigned blocks = (unsigned)((std::min<long long>((long long)c->npts * 32, cap) + CS_WARPS - 1) / CS_WARPS);
        if (has_walls(c))
            k_fixup<S, true><<<blocks, site_block(), 0, c->stream>>>(src, dst, floc, c->fix_list, count, c->geom, k, fu,
                                                                     c->scale, c->inv_scale, c->seed);
        else
            k_fixup<S, false><<<blocks, site_block(), 0, c->stream>>>(src, dst, floc, c->fix_list, count, c->geom, k, fu,
                                                                      c->scale, c->inv_scale, c->seed);
        c->launches++;
    }
    c->seed = c->seed * 747796405u + 2891336453u;  // next step's rounding seed
    return cudaGetLastError();
}

cudaError_t launch_collide(lb_ctx* c) {
    switch (c->prec) {
        case LB_F64: return collide_t<double>(c);
        case LB_F32: return collide_t<float>(c);
        case LB_F16S: return collide_t<__half>(c);
        default: return collide_t<__nv_bfloat16>(c);
    }
}

}  // namespace lbk
