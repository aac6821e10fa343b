// lb_batch.cu -- many independent lattices (replicas of uneven sizes)
// advanced together: every phase of a time step is one launch over all
// replicas, the collide+stream phase a persistent kernel that walks a work
// list of 4-tile groups spanning every replica, and a CUDA graph replays the
// step so a short lattice costs no launch overhead.  The launch shape of
// the persistent kernel is picked by timing candidates on the batch itself.
//
// The method per replica is exactly that of lb_step (same device helpers:
// Sec. II collision, Sec. III spreading, Sec. IV colloid update).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/lb.h"
#include "lb_internal.h"
#include "lb_points.cuh"

namespace {

using namespace lbk;

constexpr int BW = 4;  // warps (tiles) per work item of the collide kernel
constexpr int SORT_EVERY = 64;  // steps between renewals of the batch's cell order
constexpr int FLAT_MIN_BLOCKS = 8;  // occupancy bound of the flat collide (blocks of 128 threads per SM)

// One replica as the batched kernels see it.
struct Entry {
    void* pop[2];              // population buffers: index = parity ^ cur0
    void* floc;
    flag_t* flags;
    void* vel;                 // velocity field written by the collide (replicas with colloids), or null
    double* pos;
    double* force;
    double* radius;
    int* mobile;
    Geom g;
    int npts;
    int cur0;                  // buffer holding the state when the batch step starts
    double coef[4];            // tau_s, tau_b, om_s, om_b
    double uf[3];              // uniform force density on fluid sites (unscaled)
    float coef_f[4];           // the same in float, for the float-arithmetic formats
    float ufs_f[3];            // uniform force in the stored units (scaled for half), float
    double inv_6pi_eta, inv_aL;
    float scale, inv_scale;
    int bin0;                  // first cell-order bin of the replica
    int nb[3];                 // its 8^3 bricks along x, y, z
    float inv_nx, inv_ny;      // 1/nx, 1/ny for the flat collide's site coordinates
};

struct Work {
    long long group_begin;     // first collide work item of the replica
    int groups_x, groups_y;    // ntx, ceil(ny / BW)
    long long pt_begin;        // first point of the replica in the batch order
};

__device__ __forceinline__ int find_entry(const long long* __restrict__ begin, int n, long long w) {
    int lo = 0, hi = n - 1;  // last e with begin[e] <= w
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// -------------------------------------------------------------- kernels
template <typename T> struct EP;  // per-replica parameters in the arithmetic type
template <> struct EP<float> {
    static __device__ __forceinline__ float coef(const Entry& E, int i) { return E.coef_f[i]; }
    static __device__ __forceinline__ float uf(const Entry& E, int a) { return E.ufs_f[a]; }
};
template <> struct EP<double> {
    static __device__ __forceinline__ double coef(const Entry& E, int i) { return E.coef[i]; }
    static __device__ __forceinline__ double uf(const Entry& E, int a) { return E.uf[a]; }
};

// pull19 of one site from a single population buffer: population i of
// element j is base[i * V + j] (32-bit indices: 19 V < 2^32 for the members
// the batch takes), so no per-population pointers are held.  A solid source
// plane selects the opposite population of the site itself.
template <typename S, bool WALLS>
__device__ __forceinline__ void pull19_base(const S* __restrict__ base, unsigned V, const Nbr& n,
                                            typename Store<S>::T f[NQ]) {
    using St = Store<S>;
    const unsigned own = n.c + n.x;
    const unsigned ym = n.c + n.dym, yp = n.c + n.dyp, zm = n.c + n.dzm, zp = n.c + n.dzp;
    const bool bm = WALLS && n.solid_zm, bp = WALLS && n.solid_zp;
    f[0] = St::ld(base, own);
    f[1] = St::ld(base, V + n.c + n.xm);
    f[2] = St::ld(base, 2 * V + n.c + n.xp);
    f[3] = St::ld(base, 3 * V + ym + n.x);
    f[4] = St::ld(base, 4 * V + yp + n.x);
    f[7] = St::ld(base, 7 * V + ym + n.xm);
    f[8] = St::ld(base, 8 * V + yp + n.xp);
    f[9] = St::ld(base, 9 * V + yp + n.xm);
    f[10] = St::ld(base, 10 * V + ym + n.xp);
    f[5] = St::ld(base, bm ? 6 * V + own : 5 * V + zm + n.x);
    f[11] = St::ld(base, bm ? 12 * V + own : 11 * V + zm + n.xm);
    f[14] = St::ld(base, bm ? 13 * V + own : 14 * V + zm + n.xp);
    f[15] = St::ld(base, bm ? 16 * V + own : 15 * V + zm + n.dym + n.x);
    f[18] = St::ld(base, bm ? 17 * V + own : 18 * V + zm + n.dyp + n.x);
    f[6] = St::ld(base, bp ? 5 * V + own : 6 * V + zp + n.x);
    f[12] = St::ld(base, bp ? 11 * V + own : 12 * V + zp + n.xp);
    f[13] = St::ld(base, bp ? 14 * V + own : 13 * V + zp + n.xm);
    f[16] = St::ld(base, bp ? 15 * V + own : 16 * V + zp + n.dyp + n.x);
    f[17] = St::ld(base, bp ? 18 * V + own : 17 * V + zp + n.dym + n.x);
}

// One site (x, y, z) of member e: pull (bounce-back at its solid planes),
// collide with the member's uniform force plus its localised force where
// the site's 8-site group is flagged (fl), store with the member's rounding
// stream; in flagged groups also the velocity for the member's colloids,
// and the consumed force is zeroed (the batch spreads it anew every step).
// The field is read through the read-only path: only this thread reads
// this site's force in the launch, and only after the read does it write.
template <typename S, bool WALLS>
__device__ __forceinline__ void batch_site(const Entry& E, int e, int x, int y, int z, unsigned fl, int parity,
                                           unsigned seed) {
    using T = typename Store<S>::T;
    constexpr bool SC = Store<S>::kScaled;
    const Geom& g = E.g;
    const unsigned V = (unsigned)g.V;
    const int b = parity ^ E.cur0;
    const S* src = (const S*)E.pop[b];
    S* dst = (S*)E.pop[b ^ 1];
    const Nbr n = neighbours(g, x, y, z);
    const unsigned site = n.c + n.x;
    T* floc = (T*)E.floc;
    if (WALLS && is_solid(g, z)) {
#pragma unroll
        for (int i = 0; i < NQ; ++i) Store<S>::st(dst, (unsigned)i * V + site, T(0), 0u);
        return;
    }
    T f[NQ], o[NQ], v3[3];
    pull19_base<S, WALLS>(src, V, n, f);  // populations first: in flight with the force loads below
    T Fx = EP<T>::uf(E, 0), Fy = EP<T>::uf(E, 1), Fz = EP<T>::uf(E, 2);
    if (fl) {
        const T s = SC ? (T)E.scale : T(1);
        Fx += __ldg(floc + site) * s;
        Fy += __ldg(floc + V + site) * s;
        Fz += __ldg(floc + 2 * V + site) * s;
    }
    Coef<T> k;
    k.tau_s = EP<T>::coef(E, 0);
    k.tau_b = EP<T>::coef(E, 1);
    k.om_s = EP<T>::coef(E, 2);
    k.om_b = EP<T>::coef(E, 3);
    collide19<T, Store<S>::kCompensate, SC, true>(f, Fx, Fy, Fz, k, o, (T)E.inv_scale, v3);
    unsigned rn = rng_seed(site ^ (unsigned)(e * 0x27d4eb2d), seed);
#pragma unroll
    for (int i = 0; i < NQ; ++i) Store<S>::st(dst, (unsigned)i * V + site, o[i], rng_next(rn));
    if (fl && E.vel) {  // v at the stencil nodes of the replica's colloids
        T* vel = (T*)E.vel;
        vel[site] = v3[0];
        vel[V + site] = v3[1];
        vel[2 * V + site] = v3[2];
    }
    if (fl) {
        floc[site] = T(0);
        floc[V + site] = T(0);
        floc[2 * V + site] = T(0);
    }
}

template <typename S>
__global__ void __launch_bounds__(BW * 32, 8)
kb_collide(const Entry* __restrict__ ent, const long long* __restrict__ gbegin, const Work* __restrict__ wk, int nrep,
           long long total_groups, int parity, const unsigned* __restrict__ step_counter) {
    using T = typename Store<S>::T;
    constexpr bool SC = Store<S>::kScaled;
    const int lane = threadIdx.x, warp = threadIdx.y;
    // rounding seed of this step (the 16-bit formats): read from device
    // memory so that graph replays draw new bits every step
    const unsigned seed = Store<S>::kScaled || sizeof(S) == 2 ? rng_seed(*step_counter, 0xB5297A4Du) : 0u;
    // each block takes a contiguous chunk of work items and walks it with
    // incremental coordinates: one search per block, none per item
    const long long chunk = (total_groups + gridDim.x - 1) / gridDim.x;
    const long long w0 = (long long)blockIdx.x * chunk;
    const long long w1 = w0 + chunk < total_groups ? w0 + chunk : total_groups;
    if (w0 >= w1) return;
    int e = find_entry(gbegin, nrep, w0);
    int tx, yg, zz;
    {
        const long long local = w0 - wk[e].group_begin;
        tx = (int)(local % wk[e].groups_x);
        const long long r = local / wk[e].groups_x;
        yg = (int)(r % wk[e].groups_y);
        zz = (int)(r / wk[e].groups_y);
    }
    for (long long w = w0; w < w1; ++w) {
        if (w > w0) {  // advance (tx, yg, z, entry)
            if (++tx == wk[e].groups_x) {
                tx = 0;
                if (++yg == wk[e].groups_y) {
                    yg = 0;
                    if (++zz == ent[e].g.nz) {
                        zz = 0;
                        ++e;
                    }
                }
            }
        }
        const Entry& E = ent[e];
        const Geom& g = E.g;
        const int y = yg * BW + warp;
        const int z = zz;
        const int x = tx * TILE_X + lane;
        if (y >= g.ny) continue;  // uniform per warp
        const unsigned tile = ((unsigned)z * (unsigned)g.ny + (unsigned)y) * (unsigned)g.ntx + (unsigned)tx;
        // the flags and the field are read through the read-only path and
        // reset below by the one warp (thread) that read them, as in k_collide
        const unsigned fl = group_flag(__ldg((const unsigned*)E.flags + tile), (unsigned)lane);
        if (x < g.nx) batch_site<S, true>(E, e, x, y, z, fl, parity, seed);
        // the first lane of each flagged group resets its flag (this warp
        // alone read the tile's flag word, in one warp-wide load)
        if (fl && (lane % GROUP_X) == 0) E.flags[tile * (TILE_X / GROUP_X) + (unsigned)lane / GROUP_X] = 0;
    }
}


// The collide over flat 32-site windows of each member's site index (x
// fastest), so that no lane idles where nx is not a multiple of 32.  Valid
// when every member has nx a multiple of 8, so that an 8-site force group
// never straddles two windows (each group's flag byte is then read and
// reset by one warp; other warps that read the same flag word use only
// their own groups' bytes), and fewer than 2^24 sites, so that the float
// division of a site index below is off by at most one before its
// correction.  Each warp walks a contiguous chunk of windows.
__device__ __forceinline__ unsigned div_small(unsigned a, unsigned d, float inv_d) {
    unsigned q = __float2uint_rz(__uint2float_rn(a) * inv_d);
    const int r = (int)(a - q * d);
    if (r < 0) --q;
    else if (r >= (int)d) ++q;
    return q;
}

template <typename S, bool WALLS>
__global__ void __launch_bounds__(128, FLAT_MIN_BLOCKS)
kb_collide_flat(const Entry* __restrict__ ent, const long long* __restrict__ wbegin, int nrep, long long total_windows,
                int parity, const unsigned* __restrict__ step_counter) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned seed = Store<S>::kScaled || sizeof(S) == 2 ? rng_seed(*step_counter, 0xB5297A4Du) : 0u;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= total_windows) return;
    // the member of window w, tracked forward as w grows
    int e = find_entry(wbegin, nrep, w);
    long long lo = wbegin[e], hi = e + 1 < nrep ? wbegin[e + 1] : total_windows;
    for (; w < total_windows; w += nwarps) {
        while (w >= hi) {  // uniform per warp
            ++e;
            lo = hi;
            hi = e + 1 < nrep ? wbegin[e + 1] : total_windows;
        }
        const Entry& E = ent[e];
        const Geom& g = E.g;
        const unsigned s = (unsigned)(w - lo) * 32u + lane;
        if (s >= (unsigned)g.V) continue;  // the ragged last window of a member
        const unsigned zy = div_small(s, (unsigned)g.nx, E.inv_nx);
        const unsigned x = s - zy * (unsigned)g.nx;
        const unsigned z = div_small(zy, (unsigned)g.ny, E.inv_ny);
        const unsigned y = zy - z * (unsigned)g.ny;
        const unsigned tile = zy * (unsigned)g.ntx + x / TILE_X;
        const unsigned fl = group_flag(__ldg((const unsigned*)E.flags + tile), x % TILE_X);
        batch_site<S, WALLS>(E, e, (int)x, (int)y, (int)z, fl, parity, seed);
        if (fl && x % GROUP_X == 0) E.flags[tile * (TILE_X / GROUP_X) + (x % TILE_X) / GROUP_X] = 0;
    }
}

// Spreading, one warp per point (the scheme of k_spread), from the stencil
// rows st[gp] written by kb_stencil / kb_update; warps take the points in
// the batch's cell order (kb_brick_*).
template <typename T>
__global__ void __launch_bounds__(256)
kb_spread(const Entry* __restrict__ ent, const long long* __restrict__ pbegin, const int* __restrict__ pent,
          const int* __restrict__ order, long long total_pts, const T* __restrict__ st) {
    const long long slot = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (slot >= total_pts) return;  // uniform per warp
    const long long gp = order[slot];
    const int lane = threadIdx.x & 31;
    const int e = pent[gp];
    const Entry& E = ent[e];
    const Geom& g = E.g;
    const int s = (int)(gp - pbegin[e]);
    const unsigned FULL = 0xffffffffu;
    const T r = lane < ST_W ? st[gp * ST_W + lane] : T(0);
    const T fl = lane < 3 ? (T)E.force[3 * s + lane] : T(0);
    const int bx = bits_int(__shfl_sync(FULL, r, 12)), by = bits_int(__shfl_sync(FULL, r, 13)),
              bz = bits_int(__shfl_sync(FULL, r, 14));
    const T F0 = __shfl_sync(FULL, fl, 0), F1 = __shfl_sync(FULL, fl, 1), F2 = __shfl_sync(FULL, fl, 2);
    const int i = lane & 3, j = (lane >> 2) & 3;
    const T wxy = __shfl_sync(FULL, r, i) * __shfl_sync(FULL, r, 4 + j);
    const int x = wrap_node(bx + i, g.nx), y = wrap_node(by + j, g.ny);
    const bool marker = (i == 0) || ((x & (GROUP_X - 1)) == 0);
    const unsigned V = (unsigned)g.V;
    T* floc = (T*)E.floc;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = (lane >> 4) + 2 * h;
        const T wz = __shfl_sync(FULL, r, 8 + k);
        const int z = wrap_node(bz + k, g.nz);
        if (is_solid(g, z)) continue;
        const T w = wxy * wz;
        const unsigned row = (unsigned)z * (unsigned)g.ny + (unsigned)y;
        const unsigned site = row * (unsigned)g.nx + (unsigned)x;
        atomicAdd(floc + site, F0 * w);
        atomicAdd(floc + V + site, F1 * w);
        atomicAdd(floc + 2 * V + site, F2 * w);
        if (marker) E.flags[row * (unsigned)g.ntx * (TILE_X / GROUP_X) + (unsigned)(x / GROUP_X)] = 1;
    }
}

// Stencil rows of every point of the batch (thread per point).
template <typename T>
__global__ void kb_stencil(const Entry* __restrict__ ent, const long long* __restrict__ pbegin, const int* __restrict__ pent,
          int nrep,
                           long long total_pts, T* __restrict__ st) {
    const long long gp = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gp >= total_pts) return;
    const int e = pent[gp];
    const Entry& E = ent[e];
    const int s = (int)(gp - pbegin[e]);
    stencil_row<T>(st + gp * ST_W, E.pos[3 * s], E.pos[3 * s + 1], E.pos[3 * s + 2]);
}

__global__ void kb_tick(unsigned* step_counter) { *step_counter += 1u; }

// Cell order of the batch's points, so that neighbouring warps of the
// spread and the interpolation work on nearby stencils of one replica: a
// counting sort on key = the replica's first bin + the 8^3 brick of the
// point within the replica.  Each replica's points stay in its own range
// of slots.  Only the order of the work depends on it, never a result
// (beyond the order of the spread's atomic additions).
constexpr int BATCH_BRICK = 8;
__global__ void kb_brick_count(const Entry* __restrict__ ent, const long long* __restrict__ pbegin,
                               const int* __restrict__ pent, long long total_pts, int* __restrict__ count,
                               int* __restrict__ key) {
    const long long gp = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gp >= total_pts) return;
    const int e = pent[gp];
    const Entry& E = ent[e];
    const int s = (int)(gp - pbegin[e]);
    int b[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) b[a] = min(max((int)E.pos[3 * s + a] / BATCH_BRICK, 0), E.nb[a] - 1);
    const int k = E.bin0 + (b[2] * E.nb[1] + b[1]) * E.nb[0] + b[0];
    key[gp] = k;
    atomicAdd(&count[k], 1);
}

__global__ void kb_brick_fill(long long total_pts, const int* __restrict__ key, const int* __restrict__ start,
                              int* __restrict__ cursor, int* __restrict__ order) {
    const long long gp = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gp >= total_pts) return;
    const int k = key[gp];
    order[start[k] + atomicAdd(&cursor[k], 1)] = (int)gp;
}

// Interpolated velocity (from the velocity field the collide wrote) at
// every colloid, one warp each (the scheme of k_interp): v[3 gp + a], FP64.
template <typename T>
__global__ void __launch_bounds__(256)
kb_interp(const Entry* __restrict__ ent, const long long* __restrict__ pbegin, const int* __restrict__ pent,
          const int* __restrict__ order, long long total_pts, const T* __restrict__ st, double* __restrict__ vout) {
    const long long slot = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (slot >= total_pts) return;  // uniform per warp
    const long long gp = order[slot];
    const int e = pent[gp];
    const Entry& E = ent[e];
    const int s = (int)(gp - pbegin[e]);
    if (!E.mobile[s]) return;  // uniform per warp
    const Geom& g = E.g;
    const int lane = threadIdx.x & 31;
    const T* vel = (const T*)E.vel;
    const unsigned FULL = 0xffffffffu;
    const T r = lane < ST_W ? st[gp * ST_W + lane] : T(0);
    const int bx = bits_int(__shfl_sync(FULL, r, 12)), by = bits_int(__shfl_sync(FULL, r, 13)),
              bz = bits_int(__shfl_sync(FULL, r, 14));
    const int i = lane & 3, j = (lane >> 2) & 3;
    const T wxy = __shfl_sync(FULL, r, i) * __shfl_sync(FULL, r, 4 + j);
    const int x = wrap_node(bx + i, g.nx), y = wrap_node(by + j, g.ny);
    const unsigned V = (unsigned)g.V;
    T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = (lane >> 4) + 2 * h;
        const T wz = __shfl_sync(FULL, r, 8 + k);
        const int z = wrap_node(bz + k, g.nz);
        if (is_solid(g, z)) continue;  // v = 0 on solid nodes
        const T w = wxy * wz;
        const unsigned site = ((unsigned)z * (unsigned)g.ny + (unsigned)y) * (unsigned)g.nx + (unsigned)x;
        acc[0] += w * vel[site];
        acc[1] += w * vel[V + site];
        acc[2] += w * vel[2 * V + site];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        for (int a = 0; a < 3; ++a) acc[a] += __shfl_xor_sync(FULL, acc[a], off);
    if (lane < 3) vout[3 * gp + lane] = (double)(lane == 0 ? acc[0] : (lane == 1 ? acc[1] : acc[2]));
}

// Colloid update of every mobile point of the batch (thread per point,
// Sec. IV with the a_L subtraction, as k_update) and the stencil row of the
// new position.
template <typename T>
__global__ void kb_update(const Entry* __restrict__ ent, const long long* __restrict__ pbegin, const int* __restrict__ pent,
          int nrep,
                          long long total_pts, const double* __restrict__ v, T* __restrict__ st) {
    const long long gp = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gp >= total_pts) return;
    const int e = pent[gp];
    const Entry& E = ent[e];
    const int s = (int)(gp - pbegin[e]);
    double P[3] = {E.pos[3 * s], E.pos[3 * s + 1], E.pos[3 * s + 2]};
    if (E.mobile[s]) {
        const double c = (recip_fp64(E.radius[s]) - E.inv_aL) * E.inv_6pi_eta;
        const int nn[3] = {E.g.nx, E.g.ny, E.g.nz};
        for (int a = 0; a < 3; ++a) {
            const double L = (double)nn[a];
            double r = P[a] + v[3 * gp + a] + E.force[3 * s + a] * c;
            if (r < 0.0) r += L;
            else if (r >= L) r -= L;
            if (!(r >= 0.0 && r < L)) {  // moved by a period or more
                r = r - L * floor(r / L);
                if (r >= L || r < 0.0) r = 0.0;
            }
            P[a] = r;
            E.pos[3 * s + a] = r;
        }
    }
    stencil_row<T>(st + gp * ST_W, P[0], P[1], P[2]);
}

}  // namespace

struct lb_batch {
    int n;
    int prec;
    std::vector<lb_ctx*> ctx;
    cudaStream_t user_stream;
    cudaStream_t stream;       // private stream: graphs cannot capture the legacy stream
    cudaEvent_t ev_in, ev_out;
    Entry* d_ent;
    long long* d_gbegin;
    long long* d_pbegin;
    Work* d_work;
    long long total_groups, total_pts, n_mobile;
    int blocks;                // persistent grid of the collide kernel
    unsigned* d_step;          // step counter seeding the stochastic rounding
    int* d_pent;               // member of every point of the batch
    int* d_order;              // the points in cell order (slot -> point)
    int* d_sort;               // counting-sort workspace: count, cursor, start, scan sums, keys
    long long total_bins;      // cell-order bins of all members
    int steps_since_sort;
    bool flat;                 // the flat collide applies (every nx % 8 == 0, V < 2^24)
    bool walls;                // some member has solid planes
    long long* d_wbegin;       // first 32-site window of every member (flat collide)
    long long total_windows;
    void* d_st;                // stencil rows of every point (ST_W elements of the arithmetic type)
    double* d_v;               // interpolated velocity of every point (3 doubles)
    int parity;                // batch steps taken since creation, mod 2
    std::vector<int> cur0;     // each member's current buffer at creation
    std::vector<unsigned> version;  // each member's configuration version at creation
    cudaGraphExec_t graph2;    // two steps (parity 0, 1)
    bool graph_ready;
    long long launches;
    std::string err;
};

namespace {

lb_status bfail(lb_batch* b, lb_status s, const std::string& m) {
    if (b) b->err = m;
    return s;
}

#define LB_BCUDA(call, where)                                                                     \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA,           \
                         std::string(where) + ": " + cudaGetErrorString(e_));                     \
    } while (0)

// Launch the phases of one step (parity p) on the batch stream: spread
// (from the stencil rows), collide (writing v at the colloids' stencil
// nodes and zeroing the consumed field), interpolation, colloid update
// (which writes the next stencil rows), and the rounding-seed counter of
// the 16-bit formats.
template <typename S>
cudaError_t launch_step(lb_batch* b, int p, int blocks) {
    using T = typename Store<S>::T;
    const unsigned wblocks = (unsigned)((b->total_pts + 7) / 8);      // warp per point
    const unsigned tblocks = (unsigned)((b->total_pts + 127) / 128);  // thread per point
    T* st = (T*)b->d_st;
    if (b->total_pts > 0)
        kb_spread<T><<<wblocks, 256, 0, b->stream>>>(b->d_ent, b->d_pbegin, b->d_pent, b->d_order, b->total_pts, st);
    if (b->flat && b->walls)
        kb_collide_flat<S, true><<<blocks, 128, 0, b->stream>>>(b->d_ent, b->d_wbegin, b->n, b->total_windows, p,
                                                                b->d_step);
    else if (b->flat)
        kb_collide_flat<S, false><<<blocks, 128, 0, b->stream>>>(b->d_ent, b->d_wbegin, b->n, b->total_windows, p,
                                                                 b->d_step);
    else
        kb_collide<S><<<blocks, dim3(32, BW), 0, b->stream>>>(b->d_ent, b->d_gbegin, b->d_work, b->n, b->total_groups,
                                                              p, b->d_step);
    if (b->n_mobile > 0) {
        kb_interp<T><<<wblocks, 256, 0, b->stream>>>(b->d_ent, b->d_pbegin, b->d_pent, b->d_order, b->total_pts, st,
                                                     b->d_v);
        kb_update<T><<<tblocks, 128, 0, b->stream>>>(b->d_ent, b->d_pbegin, b->d_pent, b->n, b->total_pts, b->d_v, st);
    }
    if (sizeof(S) == 2) kb_tick<<<1, 1, 0, b->stream>>>(b->d_step);
    return cudaGetLastError();
}

// The batch's cell order (5 kernel launches): counts per bin, their
// exclusive scan, and the fill of the order.
cudaError_t launch_sort(lb_batch* b) {
    if (b->total_pts == 0) return cudaSuccess;
    const long long nb = b->total_bins;
    int* count = b->d_sort;
    int* cursor = count + nb;
    int* start = cursor + nb;
    int* bsum = start + nb + 1;
    int* key = bsum + scan_ws_ints(nb);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * 2 * (size_t)nb, b->stream);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((b->total_pts + 255) / 256);
    kb_brick_count<<<blocks, 256, 0, b->stream>>>(b->d_ent, b->d_pbegin, b->d_pent, b->total_pts, count, key);
    e = scan_exclusive(count, nb, start, bsum, b->stream);
    if (e != cudaSuccess) return e;
    kb_brick_fill<<<blocks, 256, 0, b->stream>>>(b->total_pts, key, start, cursor, b->d_order);
    b->launches += 5;
    b->steps_since_sort = 0;
    return cudaGetLastError();
}

// Stencil rows of the members' current positions (before a batch step).
template <typename S>
cudaError_t launch_stencils(lb_batch* b) {
    using T = typename Store<S>::T;
    if (b->total_pts == 0) return cudaSuccess;
    kb_stencil<T><<<(unsigned)((b->total_pts + 127) / 128), 128, 0, b->stream>>>(b->d_ent, b->d_pbegin, b->d_pent, b->n,
                                                                                b->total_pts, (T*)b->d_st);
    return cudaGetLastError();
}

cudaError_t launch_stencils_any(lb_batch* b) {
    switch (b->prec) {
        case LB_F64: return launch_stencils<double>(b);
        case LB_F32: return launch_stencils<float>(b);
        case LB_F16S: return launch_stencils<__half>(b);
        default: return launch_stencils<__nv_bfloat16>(b);
    }
}

cudaError_t launch_step_any(lb_batch* b, int p, int blocks) {
    switch (b->prec) {
        case LB_F64: return launch_step<double>(b, p, blocks);
        case LB_F32: return launch_step<float>(b, p, blocks);
        case LB_F16S: return launch_step<__half>(b, p, blocks);
        default: return launch_step<__nv_bfloat16>(b, p, blocks);
    }
}

template <typename S>
cudaError_t launch_collide_only(lb_batch* b, int blocks) {
    if (b->flat && b->walls)
        kb_collide_flat<S, true><<<blocks, 128, 0, b->stream>>>(b->d_ent, b->d_wbegin, b->n, b->total_windows,
                                                                b->parity, b->d_step);
    else if (b->flat)
        kb_collide_flat<S, false><<<blocks, 128, 0, b->stream>>>(b->d_ent, b->d_wbegin, b->n, b->total_windows,
                                                                 b->parity, b->d_step);
    else
        kb_collide<S><<<blocks, dim3(32, BW), 0, b->stream>>>(b->d_ent, b->d_gbegin, b->d_work, b->n, b->total_groups,
                                                              b->parity, b->d_step);
    return cudaGetLastError();
}

cudaError_t launch_collide_any(lb_batch* b, int blocks) {
    switch (b->prec) {
        case LB_F64: return launch_collide_only<double>(b, blocks);
        case LB_F32: return launch_collide_only<float>(b, blocks);
        case LB_F16S: return launch_collide_only<__half>(b, blocks);
        default: return launch_collide_only<__nv_bfloat16>(b, blocks);
    }
}

int launches_per_step(const lb_batch* b) {
    return 1 + (b->total_pts > 0 ? 1 : 0) + (b->n_mobile > 0 ? 2 : 0) + (b->prec >= LB_F16S ? 1 : 0);
}

}  // namespace

extern "C" {

lb_status lb_batch_create(lb_batch** out, int n, lb_ctx* const* ctxs, void* stream) {
    if (!out || n < 1 || !ctxs) return LB_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i] || ctxs[i]->prec != ctxs[0]->prec || ctxs[i]->device != ctxs[0]->device) return LB_ERR_ARG;
    lb_batch* b = new (std::nothrow) lb_batch();
    if (!b) return LB_ERR_OOM;
    b->n = n;
    b->prec = ctxs[0]->prec;
    b->ctx.assign(ctxs, ctxs + n);
    b->user_stream = (cudaStream_t)stream;
    b->parity = 0;
    std::vector<Entry> ent(n);
    std::vector<long long> gbegin(n), pbegin(n);
    std::vector<Work> work(n);
    long long groups = 0, pts = 0, mob = 0, bins = 0, windows = 0;
    std::vector<long long> wbegin(n);
    bool flat = true, walls = false;
    for (int i = 0; i < n; ++i) {
        lb_ctx* c = ctxs[i];
        Entry& E = ent[i];
        E.pop[0] = c->f[0];
        E.pop[1] = c->f[1];
        E.floc = c->floc;
        E.flags = c->flags;
        E.vel = nullptr;
        if (c->n_mobile > 0) {
            const cudaError_t ev = lbk::ensure_velocity_field(c);
            if (ev != cudaSuccess) {
                delete b;
                return ev == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA;
            }
            E.vel = c->vel;
        }
        E.pos = c->pos;
        E.force = c->force;
        E.radius = c->radius;
        E.mobile = c->mobile;
        E.g = c->geom;
        E.npts = c->npts;
        E.cur0 = c->cur;
        b->cur0.push_back(c->cur);
        b->version.push_back(c->version);
        E.coef[0] = c->tau_s;
        E.coef[1] = c->tau_b;
        E.coef[2] = 1.0 / (c->tau_s + 0.5);
        E.coef[3] = 1.0 / (c->tau_b + 0.5);
        const UForce<double> u = uniform_force<double>(c);
        for (int a = 0; a < 3; ++a) {
            E.uf[a] = u.F[a];
            E.ufs_f[a] = (float)(u.F[a] * (double)c->scale);
        }
        for (int a = 0; a < 4; ++a) E.coef_f[a] = (float)E.coef[a];
        E.inv_6pi_eta = 1.0 / (6.0 * M_PI * (c->tau_s / 3.0));
        E.inv_aL = isinf(c->a_L) ? 0.0 : 1.0 / c->a_L;
        E.scale = c->scale;
        E.inv_scale = c->inv_scale;
        for (int a = 0; a < 3; ++a) {
            const int len = a == 0 ? c->geom.nx : (a == 1 ? c->geom.ny : c->geom.nz);
            E.nb[a] = (len + BATCH_BRICK - 1) / BATCH_BRICK;
        }
        E.bin0 = (int)bins;
        bins += (long long)E.nb[0] * E.nb[1] * E.nb[2];
        E.inv_nx = 1.0f / (float)c->geom.nx;
        E.inv_ny = 1.0f / (float)c->geom.ny;
        flat = flat && c->geom.nx % GROUP_X == 0 && c->geom.V < (1LL << 24);
        walls = walls || has_walls(c);
        wbegin[i] = windows;
        windows += (c->geom.V + 31) / 32;
        work[i].groups_x = c->geom.ntx;
        work[i].groups_y = (c->geom.ny + BW - 1) / BW;
        work[i].group_begin = groups;
        work[i].pt_begin = pts;
        gbegin[i] = groups;
        pbegin[i] = pts;
        groups += (long long)work[i].groups_x * work[i].groups_y * c->geom.nz;
        pts += c->npts;
        mob += c->n_mobile;
    }
    b->total_groups = groups;
    b->total_pts = pts;
    b->n_mobile = mob;
    b->total_bins = bins;
    b->steps_since_sort = SORT_EVERY;  // the first step sorts
    b->flat = flat;
    b->walls = walls;
    b->total_windows = windows;
    // untuned: the flat collide 8 blocks per SM, the tiled one a block per item
    b->blocks = flat ? 152 * 8 : (int)std::min<long long>(std::max<long long>(groups, 1), 0x7fffffffLL);
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ent, sizeof(Entry) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_gbegin, sizeof(long long) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_pbegin, sizeof(long long) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_work, sizeof(Work) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_wbegin, sizeof(long long) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_step, sizeof(unsigned));
    if (e == cudaSuccess && pts > 0)
        e = cudaMalloc(&b->d_st, lbk::arith_bytes(b->prec) * ST_W * (size_t)pts);
    if (e == cudaSuccess && pts > 0) e = cudaMalloc(&b->d_v, sizeof(double) * 3 * (size_t)pts);
    if (e == cudaSuccess && pts > 0) e = cudaMalloc(&b->d_order, sizeof(int) * (size_t)pts);
    if (e == cudaSuccess && pts > 0)
        e = cudaMalloc(&b->d_sort, sizeof(int) * ((size_t)(3 * bins + 1) + scan_ws_ints(bins) + (size_t)pts));
    if (e == cudaSuccess && pts > 0) {
        std::vector<int> pent((size_t)pts);
        for (int i = 0; i < n; ++i)
            for (long long q = pbegin[i]; q < pbegin[i] + ctxs[i]->npts; ++q) pent[(size_t)q] = i;
        e = cudaMalloc(&b->d_pent, sizeof(int) * (size_t)pts);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_pent, pent.data(), sizeof(int) * (size_t)pts, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(b->d_step, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_ent, ent.data(), sizeof(Entry) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_gbegin, gbegin.data(), sizeof(long long) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_pbegin, pbegin.data(), sizeof(long long) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_work, work.data(), sizeof(Work) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_wbegin, wbegin.data(), sizeof(long long) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        lb_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA;
    }
    *out = b;
    return LB_OK;
}

void lb_batch_destroy(lb_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph_ready) cudaGraphExecDestroy(b->graph2);
    cudaFree(b->d_ent);
    cudaFree(b->d_gbegin);
    cudaFree(b->d_pbegin);
    cudaFree(b->d_work);
    cudaFree(b->d_wbegin);
    cudaFree(b->d_step);
    cudaFree(b->d_st);
    cudaFree(b->d_v);
    cudaFree(b->d_pent);
    cudaFree(b->d_order);
    cudaFree(b->d_sort);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char* lb_batch_last_error(const lb_batch* b) { return b ? b->err.c_str() : ""; }

lb_status lb_batch_tune(lb_batch* b, int* blocks_out) {
    if (!b) return LB_ERR_ARG;
    // Whole trial steps are timed (spread, collide + stream, interpolation,
    // update), since the collide's best grid depends on the phases around
    // it.  A trial does not advance the batch: the parity is not flipped,
    // so every trial reads the same current population buffers and writes
    // the spare ones; the collide zeroes the force it consumed; the
    // positions and the rounding counter the trials move are saved first
    // and put back after the last trial.  A spread field of a query is
    // cleared first (the next step spreads again).
    for (lb_ctx* c : b->ctx) {
        if (c->field_ready) {
            LB_BCUDA(lbk::launch_clear_field(c), "clear force field");
            c->field_ready = false;
        }
        LB_BCUDA(cudaStreamSynchronize(c->stream), "member stream");
    }
    double* saved_pos = nullptr;
    unsigned* saved_step = nullptr;
    LB_BCUDA(cudaMalloc(&saved_step, sizeof(unsigned)), "tuner scratch");
    if (b->total_pts > 0) {
        cudaError_t e = cudaMalloc(&saved_pos, sizeof(double) * 3 * (size_t)b->total_pts);
        if (e != cudaSuccess) {
            cudaFree(saved_step);
            return bfail(b, LB_ERR_OOM, "tuner scratch");
        }
    }
    const auto copy_positions = [&](bool save) -> cudaError_t {
        size_t off = 0;
        for (lb_ctx* c : b->ctx) {
            if (c->npts == 0) continue;
            const size_t bytes = sizeof(double) * 3 * (size_t)c->npts;
            cudaError_t e = save ? cudaMemcpyAsync(saved_pos + off, c->pos, bytes, cudaMemcpyDeviceToDevice, b->stream)
                                 : cudaMemcpyAsync(c->pos, saved_pos + off, bytes, cudaMemcpyDeviceToDevice, b->stream);
            if (e != cudaSuccess) return e;
            off += 3 * (size_t)c->npts;
        }
        return save ? cudaMemcpyAsync(saved_step, b->d_step, sizeof(unsigned), cudaMemcpyDeviceToDevice, b->stream)
                    : cudaMemcpyAsync(b->d_step, saved_step, sizeof(unsigned), cudaMemcpyDeviceToDevice, b->stream);
    };
    cudaError_t err = copy_positions(true);
    // the stencil rows and the cell order of the current positions
    if (err == cudaSuccess) err = launch_stencils_any(b);
    if (err == cudaSuccess && b->total_pts > 0) err = launch_sort(b);
    int best = b->blocks;
    float best_ms = 1e30f;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (err == cudaSuccess) err = cudaEventCreate(&t0);
    if (err == cudaSuccess) err = cudaEventCreate(&t1);
    // candidates: persistent grids of 2-16 blocks per SM (contiguous chunks of
    // work per block or warp), and for the tiled collide one block per work
    // item (no persistence)
    const long long per_sm_tiled[] = {2, 4, 8, 16, 0};
    const long long per_sm_flat[] = {4, 6, 8, 12, 16};
    const long long* per_sm = b->flat ? per_sm_flat : per_sm_tiled;
    const long long items = b->flat ? (b->total_windows + 3) / 4 : b->total_groups;
    for (int ci = 0; ci < 5 && err == cudaSuccess; ++ci) {
        const long long k = per_sm[ci];
        const long long want = k ? 152LL * k : std::min<long long>(items, 0x7fffffffLL);
        const int blocks = (int)std::min<long long>(want, std::max<long long>(1, items));
        err = launch_step_any(b, b->parity, blocks);  // warm
        if (err == cudaSuccess) err = cudaEventRecord(t0, b->stream);
        for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = launch_step_any(b, b->parity, blocks);
        if (err == cudaSuccess) err = cudaEventRecord(t1, b->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, t0, t1);
        if (err == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = blocks;
        }
        b->launches += 4LL * launches_per_step(b);
    }
    if (err == cudaSuccess) err = copy_positions(false);
    if (err == cudaSuccess) err = launch_stencils_any(b);
    if (err == cudaSuccess) err = cudaStreamSynchronize(b->stream);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(saved_pos);
    cudaFree(saved_step);
    if (err != cudaSuccess) return bfail(b, LB_ERR_CUDA, std::string("lb_batch_tune: ") + cudaGetErrorString(err));
    if (best != b->blocks && b->graph_ready) {
        cudaGraphExecDestroy(b->graph2);
        b->graph_ready = false;
    }
    b->blocks = best;
    if (blocks_out) *blocks_out = best;
    return LB_OK;
}

lb_status lb_batch_step(lb_batch* b, int nsteps) {
    if (!b) return LB_ERR_ARG;
    if (nsteps < 0) return bfail(b, LB_ERR_ARG, "lb_batch_step: nsteps < 0");
    if (nsteps == 0) return LB_OK;
    for (int i = 0; i < b->n; ++i) {
        lb_ctx* c = b->ctx[i];
        if (c->version != b->version[i] || c->cur != (b->cur0[i] ^ b->parity))
            return bfail(b, LB_ERR_STATE,
                         "lb_batch_step: a member was reconfigured or stepped on its own since lb_batch_create");
    }
    // order after the caller's stream and the member contexts' work
    LB_BCUDA(cudaEventRecord(b->ev_in, b->user_stream), "event record");
    LB_BCUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0), "stream wait");
    for (lb_ctx* c : b->ctx) {
        if (c->stream != b->user_stream) {
            LB_BCUDA(cudaEventRecord(b->ev_in, c->stream), "event record");
            LB_BCUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0), "stream wait");
        }
        if (c->field_ready) {  // forces already spread by a query: clear, the step spreads again
            LB_BCUDA(lbk::launch_clear_field(c), "clear force field");
            LB_BCUDA(cudaEventRecord(b->ev_in, c->stream), "event record");
            LB_BCUDA(cudaStreamWaitEvent(b->stream, b->ev_in, 0), "stream wait");
            c->field_ready = false;
        }
    }
    // the positions may have been set since the last batch step
    LB_BCUDA(launch_stencils_any(b), "stencil kernel");
    b->launches += b->total_pts > 0 ? 1 : 0;
    if (!b->graph_ready && nsteps >= 2) {
        cudaGraph_t g;
        LB_BCUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t e = launch_step_any(b, 0, b->blocks);
        if (e == cudaSuccess) e = launch_step_any(b, 1, b->blocks);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess)
            return bfail(b, LB_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        e = cudaGraphInstantiate(&b->graph2, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(b, LB_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        b->graph_ready = true;
    }
    // The graph holds two steps starting at parity 0: a batch at odd parity
    // takes one plain step first.
    // The cell order is renewed every SORT_EVERY steps (outside the graph).
    int done = 0;
    while (done < nsteps) {
        if (b->steps_since_sort >= SORT_EVERY) LB_BCUDA(launch_sort(b), "cell order kernels");
        if (b->graph_ready && b->parity == 0 && nsteps - done >= 2) {
            LB_BCUDA(cudaGraphLaunch(b->graph2, b->stream), "graph launch");
            done += 2;
            b->steps_since_sort += 2;
        } else {
            LB_BCUDA(launch_step_any(b, b->parity, b->blocks), "batched step");
            b->parity ^= 1;
            done += 1;
            b->steps_since_sort += 1;
        }
    }
    b->launches += (long long)nsteps * launches_per_step(b);
    for (lb_ctx* c : b->ctx) {
        c->cur ^= (nsteps & 1);
        c->field_ready = false;
    }
    LB_BCUDA(cudaEventRecord(b->ev_out, b->stream), "event record");
    LB_BCUDA(cudaStreamWaitEvent(b->user_stream, b->ev_out, 0), "stream wait");
    for (lb_ctx* c : b->ctx)
        if (c->stream != b->user_stream) LB_BCUDA(cudaStreamWaitEvent(c->stream, b->ev_out, 0), "stream wait");
    return LB_OK;
}

lb_status lb_batch_info(const lb_batch* b, long long* sites, long long* points, int* blocks, long long* launches) {
    if (!b) return LB_ERR_ARG;
    long long s = 0;
    for (lb_ctx* c : b->ctx) s += c->geom.V;
    if (sites) *sites = s;
    if (points) *points = b->total_pts;
    if (blocks) *blocks = b->blocks;
    if (launches) *launches = b->launches;
    return LB_OK;
}

}  // extern "C"
