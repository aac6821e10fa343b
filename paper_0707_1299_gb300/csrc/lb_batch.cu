// lb_batch.cu -- many independent lattices (replicas of uneven sizes)
// advanced together, one persistent cooperative launch per time step over
// all replicas.  Inside the launch:
//   (every 64 steps) the cell order of all points -- a counting sort between
//     grid-wide barriers;
//   (first step of a call, when the force fields are not spread) stencil
//     rows of the current positions and the spread, then a grid barrier;
//   then a work queue that the blocks drain from one counter: the collide +
//   stream of every replica in chunks, replica after replica (writing the
//   fluid velocity at the colloids' stencil nodes, zeroing the consumed
//   force), then the point items (interpolation, colloid update and the
//   spread of the forces at the new positions for the next step), each of
//   which waits until the collide chunks of its own replica are done.  No
//   block idles at a barrier while others finish their share of the collide.
// Every wait is bounded; a wait that runs out sets an error flag and the
// kernel returns (lb_batch_synchronize reports LB_ERR_TIMEOUT).  Two steps
// (the two buffer parities) are replayed from a CUDA graph.  The grid
// (blocks per SM) is picked by timing candidates on the batch itself.
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

constexpr int BW = 4;               // warps (tiles) per work item of the tiled collide
constexpr int BT = BW * 32;         // threads per block of the persistent kernel
constexpr int SORT_EVERY = 64;      // steps between renewals of the batch's cell order
// Occupancy bound of the persistent kernel (blocks of 128 threads per SM).
// With the work queue, 8 (64 registers) measured fastest on the 64-replica
// FP32 batch: 1.513 ms a step against 1.521 at 7 and 1.569 at 6 (with grid
// barriers between the phases 6 had been fastest).  The FP64 kernel spills
// at 64 registers and keeps 6.
template <typename S>
constexpr int min_blocks() {
    return sizeof(typename Store<S>::T) == 8 ? 6 : 8;
}
constexpr long long DEFAULT_WAIT = 1LL << 22;  // polls of a wait (~1 s) before it gives up
// Collide chunks: about CHUNKS_PER_BLOCK per resident block, so that the
// tail (the last chunk a block takes) stays short, in a power of two of
// 32-site windows (flat walk) or 4-tile groups (tiled walk) between the
// bounds below.  On the 64-replica batch (53.8 M sites, 912 blocks: 256
// windows a chunk) 64, 128 and 512 windows measured 1.670, 1.644 and 1.638
// ms a step against 1.626 (fewer chunks: longer tail; more: more queue
// traffic); with 8192-site chunks a 12-replica batch (10.5 M sites) left
// 1.4 chunks a block and took 0.438 ms a step.
constexpr int CHUNKS_PER_BLOCK = 6;
constexpr int CHUNK_MIN = 16, CHUNK_MAX = 256;
constexpr int NPB = 4 * (BT / 32);  // points of a block's point item

// Barrier, work-queue and step state of a batch, in device memory.  The
// queue counters return to zero at the end of every launch (the last block
// to leave resets them).
struct BatchCtl {
    unsigned count;      // blocks arrived at the current barrier
    unsigned gen;        // barrier generation
    int err;             // 1: a wait ran out
    int init;            // 1: spread the forces at the current positions before the collide
    unsigned since_sort; // steps since the cell order was renewed
    unsigned step;       // step counter seeding the stochastic rounding of the 16-bit formats
    long long limit;     // polls of a wait
    unsigned next;       // next work item of the queue
    unsigned exits;      // blocks that have left the launch
};

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
    int groups_x, groups_y;    // ntx, ceil(ny / BW): the tiled walk's 4-tile groups per plane
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
        T lx, ly, lz;
        field_ldg(floc, site, lx, ly, lz);
        Fx += lx * s;
        Fy += ly * s;
        Fz += lz * s;
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
    if (fl && E.vel) field_st((T*)E.vel, site, v3[0], v3[1], v3[2]);  // v at the replica's colloids' nodes
    if (fl) field_st(floc, site, T(0), T(0), T(0));
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



// ------------------------------------------------------ grid barrier
// All blocks of the (cooperative, co-resident) grid meet here.  Thread 0 of
// each block arrives with a fenced atomic; the last to arrive resets the
// count and opens the next generation.  The others poll the generation at
// most ctl->limit times (with a short sleep between polls); a wait that runs
// out sets the error flag and the block leaves the kernel.  Returns false
// (in every thread of the block) after a timeout.
__device__ __forceinline__ bool grid_sync(BatchCtl* ctl, long long limit) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = &ctl->gen;
        const unsigned g0 = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&ctl->count, 0u);
            __threadfence();
            atomicAdd(&ctl->gen, 1u);
        } else {
            long long polls = 0;
            while (*vgen == g0) {
                if (polls++ >= limit) {
                    ok = 0;
                    atomicOr(&ctl->err, 1);
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

// Everything the persistent kernel reads.
struct StepArgs {
    const Entry* ent;
    int nrep;
    // tiled collide walk
    const Work* work;
    int chunk;              // windows (flat walk) or 4-tile groups (tiled walk) a collide chunk
    // the work queue: segment k holds items [sbegin[k], sbegin[k + 1]) of one
    // member, collide chunks (skind[k] = 0) or point items (1); member e has
    // nchunk[e] chunks in all, done[e] counts the finished ones
    const long long* sbegin;
    const int* smember;
    const int* skind;
    int nseg;
    long long total_items;
    const int* nchunk;
    unsigned* done;
    // points
    const long long* pbegin;
    const int* pent;
    int* order;
    long long total_pts, n_mobile;
    void* st;               // stencil rows (ST_W elements of the arithmetic type per point)
    // cell order
    int* sort_ws;           // count[nb], cursor[nb], start[nb + 1], key[total_pts]
    long long total_bins;
    BatchCtl* ctl;
};

// The point view of point gp of the batch.
template <typename T>
struct BatchPoints {
    const Entry* ent;
    const long long* pbegin;
    const int* pent;
    __device__ __forceinline__ PointView<T> view(long long gp) const {
        const int e = pent[gp];
        const Entry& E = ent[e];
        PointView<T> P;
        P.g = E.g;
        P.floc = (T*)E.floc;
        P.flags = E.flags;
        P.vel = (const T*)E.vel;
        P.pos = E.pos;
        P.force = E.force;
        P.radius = E.radius;
        P.mobile = E.mobile;
        P.inv_aL = E.inv_aL;
        P.inv_6pi_eta = E.inv_6pi_eta;
        P.s = (int)(gp - pbegin[e]);
        return P;
    }
    __device__ __forceinline__ const float* y(long long) const { return nullptr; }
};

// Cell order of the batch's points (a counting sort on key = the member's
// first bin + the 8^3 brick of the point within the member), so that
// neighbouring warps of the point phase work on nearby stencils of one
// replica.  Only the order of the work depends on it, never a result
// (beyond the order of the spread's atomic additions).  Four barriers.
constexpr int BATCH_BRICK = 8;
__device__ bool sort_points(const StepArgs& a, long long limit) {
    const long long nb = a.total_bins;
    int* count = a.sort_ws;
    int* cursor = count + nb;
    int* start = cursor + nb;
    int* key = start + nb + 1;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    for (long long i = tid; i < 2 * nb; i += nthreads) count[i] = 0;  // count and cursor
    if (!grid_sync(a.ctl, limit)) return false;
    for (long long gp = tid; gp < a.total_pts; gp += nthreads) {
        const int e = a.pent[gp];
        const Entry& E = a.ent[e];
        const int s = (int)(gp - a.pbegin[e]);
        int b[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) b[d] = min(max((int)E.pos[3 * s + d] / BATCH_BRICK, 0), E.nb[d] - 1);
        const int k = E.bin0 + (b[2] * E.nb[1] + b[1]) * E.nb[0] + b[0];
        key[gp] = k;
        atomicAdd(&count[k], 1);
    }
    if (!grid_sync(a.ctl, limit)) return false;
    if (blockIdx.x == 0) {  // exclusive scan of the counts by one block: a chunk a thread
        __shared__ int part[BT + 1];
        const long long chunk = (nb + BT - 1) / BT;
        const long long c0 = threadIdx.x * chunk, c1 = min(c0 + chunk, nb);
        int sum = 0;
        for (long long i = c0; i < c1; ++i) sum += count[i];
        part[threadIdx.x] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
            for (int t = 0; t < BT; ++t) {
                const int v = part[t];
                part[t] = run;
                run += v;
            }
            part[BT] = run;
        }
        __syncthreads();
        int run = part[threadIdx.x];
        for (long long i = c0; i < c1; ++i) {
            start[i] = run;
            run += count[i];
        }
        if (threadIdx.x == 0) start[nb] = part[BT];
    }
    if (!grid_sync(a.ctl, limit)) return false;
    for (long long gp = tid; gp < a.total_pts; gp += nthreads) {
        const int k = key[gp];
        a.order[start[k] + atomicAdd(&cursor[k], 1)] = (int)gp;
    }
    return grid_sync(a.ctl, limit);
}

// Collide chunk c of replica e, tiled walk (any geometry): a.chunk
// 4-tile groups of the replica in order; warp w of the block takes row
// y = 4 yg + w of a group.
template <typename S>
__device__ __forceinline__ void tiled_chunk(const StepArgs& a, int e, long long c, int parity, unsigned seed) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Entry& E = a.ent[e];
    const Geom& g = E.g;
    const Work& W = a.work[e];
    const long long n_groups = (long long)W.groups_x * W.groups_y * g.nz;
    const long long i1 = min((c + 1) * a.chunk, n_groups);
    for (long long it = c * a.chunk; it < i1; ++it) {
        const int tx = (int)(it % W.groups_x);
        const long long r = it / W.groups_x;
        const int y = (int)(r % W.groups_y) * BW + warp;
        const int z = (int)(r / W.groups_y);
        const int x = tx * TILE_X + lane;
        if (y >= g.ny) continue;  // uniform per warp
        const unsigned tile = ((unsigned)z * (unsigned)g.ny + (unsigned)y) * (unsigned)g.ntx + (unsigned)tx;
        // the flags and the field are read through the read-only path and
        // reset below by the one warp (thread) that read them, as in k_collide
        const unsigned fl = group_flag(__ldg((const unsigned*)E.flags + tile), (unsigned)lane);
        if (x < g.nx) batch_site<S, true>(E, e, x, y, z, fl, parity, seed);
        if (fl && (lane % GROUP_X) == 0) E.flags[tile * (TILE_X / GROUP_X) + (unsigned)lane / GROUP_X] = 0;
    }
}

// Collide chunk c of replica e, flat walk: a.chunk 32-site windows of the
// replica's site index (see div_small), window k of the chunk to warp k % 4.
template <typename S, bool WALLS>
__device__ __forceinline__ void flat_chunk(const StepArgs& a, int e, long long c, int parity, unsigned seed) {
    const unsigned lane = threadIdx.x & 31u;
    const Entry& E = a.ent[e];
    const Geom& g = E.g;
    const long long w0 = c * a.chunk;
    const long long w1 = min(w0 + a.chunk, ((long long)g.V + 31) / 32);
    for (long long w = w0 + (threadIdx.x >> 5); w < w1; w += BT / 32) {
        const unsigned s = (unsigned)w * 32u + lane;
        if (s >= (unsigned)g.V) continue;  // the ragged last window of a replica
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

// Thread 0 of a block: wait (bounded) until every collide chunk of the
// members of the points in cell-order slots [p0, p1) is done, then fence
// so that the block reads their velocity fields and writes their force
// fields after the collide.  False after a timeout (error flag set).
__device__ bool wait_replicas(const StepArgs& a, long long p0, long long p1, long long limit) {
    int last = -1;
    for (long long p = p0; p < p1; ++p) {
        const int e = a.pent[a.order[p]];
        if (e == last) continue;
        last = e;
        const unsigned need = (unsigned)a.nchunk[e];
        const volatile unsigned* d = a.done + e;
        long long polls = 0;
        while (*d < need) {
            if (polls++ >= limit) {
                atomicOr(&a.ctl->err, 1);
                return false;
            }
            __nanosleep(64);
        }
    }
    __threadfence();
    return true;
}

// One time step of every member (buffer parity `parity`).  The state flags
// (init, since_sort, step, limit) are read by every block at its start and
// rewritten, with the queue counters reset, by the last block to leave, so
// all blocks of a launch see the same values.  Work items come from one
// counter in queue order: the collide chunks, member after member, then the
// point items, member after member (a member's slots of the cell order,
// which the sort keeps member after member).  A block fetches its next item
// while it works on the current one.  No wait can stall for good: a point
// item waits only for chunks, which all come before it in the queue, and a
// block holds a fetched chunk only while its current item is a chunk (no
// wait), so every chunk is being worked on or will be next.  (Placing a
// member's point items among later members' chunks instead, to overlap
// them with the collide, measured slower: both compete for the memory.)
template <typename S, bool FLAT, bool WALLS>
__global__ void __launch_bounds__(BT, min_blocks<S>()) kb_step(const StepArgs a, int parity) {
    using T = typename Store<S>::T;
    BatchCtl* ctl = a.ctl;
    const volatile BatchCtl* vc = ctl;
    const long long limit = vc->limit;
    const bool init = vc->init != 0 && a.total_pts > 0;
    const unsigned since = vc->since_sort;
    const bool sort_due = since >= (unsigned)SORT_EVERY && a.total_pts > 0;
    const unsigned step = vc->step;
    const unsigned seed = sizeof(S) == 2 ? rng_seed(step, 0xB5297A4Du) : 0u;
    const long long items = (a.total_pts + NPB - 1) / NPB;
    __shared__ double vsh[NPB][3];
    __shared__ unsigned s_item;
    const BatchPoints<T> src{a.ent, a.pbegin, a.pent};
    T* st = (T*)a.st;
    if (sort_due && !sort_points(a, limit)) return;
    if (init) {  // stencil rows and spread at the current positions
        for (long long q = blockIdx.x; q < items; q += gridDim.x)
            point_block<T, WALLS, false, BT / 32>(src, q * NPB, a.total_pts, a.order, st, vsh);
        if (!grid_sync(ctl, limit)) return;
    }
    if (threadIdx.x == 0) s_item = atomicAdd(&ctl->next, 1u);
    __syncthreads();
    for (;;) {
        const long long t = s_item;
        if (t >= a.total_items) break;
        unsigned t_next = 0;
        if (threadIdx.x == 0) t_next = atomicAdd(&ctl->next, 1u);  // in flight during this item
        const int k = find_entry(a.sbegin, a.nseg, t);
        const int e = a.smember[k];
        const long long j = t - a.sbegin[k];
        if (a.skind[k] == 0) {
            if (FLAT) flat_chunk<S, WALLS>(a, e, j, parity, seed);
            else tiled_chunk<S>(a, e, j, parity, seed);
            __threadfence();  // this thread's stores, device-wide, before the count
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(&a.done[e], 1u);
        } else {
            const long long p0 = a.pbegin[e] + j * NPB;
            const long long p1 = min(p0 + NPB, a.pbegin[e] + a.ent[e].npts);
            int ok = 1;
            if (threadIdx.x == 0) ok = wait_replicas(a, p0, p1, limit);
            if (!__syncthreads_and(ok)) return;
            point_block<T, WALLS, true, BT / 32>(src, p0, p1, a.order, st, vsh);
        }
        __syncthreads();
        if (threadIdx.x == 0) s_item = t_next;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctl->exits, 1u) == gridDim.x - 1) {  // every other block has left
            for (int m = 0; m < a.nrep; ++m) a.done[m] = 0;
            ctl->next = 0;
            ctl->exits = 0;
            ctl->init = 0;
            ctl->since_sort = sort_due ? 1u : since + 1u;
            ctl->step = step + 1u;
            __threadfence();
        }
    }
}

}  // namespace

struct lb_batch {
    int n;
    int prec;
    std::vector<lb_ctx*> ctx;
    cudaStream_t user_stream;
    cudaStream_t stream;       // private stream: graphs cannot capture the legacy stream
    cudaEvent_t ev_in, ev_out, ev_err;
    Entry* d_ent;
    long long* d_pbegin;
    Work* d_work;
    long long* d_sbegin;       // work-queue segments: first item, member, kind
    int* d_smember;
    int* d_skind;
    int nseg;
    long long total_items;
    int chunk;                 // windows or 4-tile groups a collide chunk
    int* d_nchunk;             // collide chunks of every member
    unsigned* d_done;          // finished collide chunks of every member (zero between launches)
    long long total_pts, n_mobile, total_bins;
    int blocks;                // grid of the persistent kernel
    int max_blocks;            // co-resident limit of that grid
    int sms;
    BatchCtl* d_ctl;
    int* h_err;                // page-locked copy of the error flag, written after every step call
    bool err_pending;          // h_err copy enqueued and not yet inspected
    int* d_pent;               // member of every point of the batch
    int* d_order;              // the points in cell order (slot -> point)
    int* d_sort;               // counting-sort workspace
    void* d_st;                // stencil rows of every point
    bool flat;                 // the flat collide applies (every nx % 8 == 0, V < 2^24)
    bool walls;                // some member has solid planes
    int parity;                // batch steps taken since creation, mod 2
    std::vector<int> cur0;     // each member's current buffer at creation
    std::vector<unsigned> version;  // each member's configuration version at creation
    cudaGraphExec_t graph2;    // two steps (parity 0, 1)
    bool graph_ready, graph_failed;
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

StepArgs step_args(const lb_batch* b) {
    StepArgs a;
    a.ent = b->d_ent;
    a.nrep = b->n;
    a.work = b->d_work;
    a.chunk = b->chunk;
    a.sbegin = b->d_sbegin;
    a.smember = b->d_smember;
    a.skind = b->d_skind;
    a.nseg = b->nseg;
    a.total_items = b->total_items;
    a.nchunk = b->d_nchunk;
    a.done = b->d_done;
    a.pbegin = b->d_pbegin;
    a.pent = b->d_pent;
    a.order = b->d_order;
    a.total_pts = b->total_pts;
    a.n_mobile = b->n_mobile;
    a.st = b->d_st;
    a.sort_ws = b->d_sort;
    a.total_bins = b->total_bins;
    a.ctl = b->d_ctl;
    return a;
}

template <typename S>
const void* step_kernel(bool flat, bool walls) {
    if (flat) return walls ? (const void*)kb_step<S, true, true> : (const void*)kb_step<S, true, false>;
    return (const void*)kb_step<S, false, true>;
}

const void* step_kernel_any(const lb_batch* b) {
    switch (b->prec) {
        case LB_F64: return step_kernel<double>(b->flat, b->walls);
        case LB_F32: return step_kernel<float>(b->flat, b->walls);
        case LB_F16S: return step_kernel<__half>(b->flat, b->walls);
        default: return step_kernel<__nv_bfloat16>(b->flat, b->walls);
    }
}

// One step (parity p): one cooperative launch of the persistent kernel, so
// that all its blocks are resident together (the barriers need it).
cudaError_t launch_step(lb_batch* b, int p, int blocks) {
    StepArgs a = step_args(b);
    void* args[2] = {&a, &p};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(BT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, step_kernel_any(b), args);
}

// Zero the force fields the members hold (where flagged) so that the next
// step spreads anew at the current positions.
cudaError_t clear_member_fields(lb_batch* b) {
    for (lb_ctx* c : b->ctx) {
        if (c->npts == 0) continue;
        cudaError_t e = lbk::launch_clear_field(c);
        if (e != cudaSuccess) return e;
        c->field_ready = false;
        b->launches++;
    }
    return cudaSuccess;
}

cudaError_t set_ctl(lb_batch* b, size_t offset, const void* v, size_t bytes) {
    return cudaMemcpyAsync((char*)b->d_ctl + offset, v, bytes, cudaMemcpyHostToDevice, b->stream);
}

// Barrier and work-queue state back to its between-launches values (after
// a launch that gave up on a wait and left it mid-way).  Synchronous.
cudaError_t reset_sync_state(lb_batch* b) {
    const unsigned zero2[2] = {0u, 0u};
    const int no = 0;
    cudaError_t e = set_ctl(b, offsetof(BatchCtl, count), zero2, sizeof(zero2));  // count, gen
    if (e == cudaSuccess) e = set_ctl(b, offsetof(BatchCtl, err), &no, sizeof(no));
    if (e == cudaSuccess) e = set_ctl(b, offsetof(BatchCtl, next), zero2, sizeof(zero2));  // next, exits
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_done, 0, sizeof(unsigned) * (size_t)b->n, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e;
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
    std::vector<long long> pbegin(n);
    std::vector<Work> work(n);
    long long pts = 0, mob = 0, bins = 0;
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
        work[i].groups_x = c->geom.ntx;
        work[i].groups_y = (c->geom.ny + BW - 1) / BW;
        pbegin[i] = pts;
        pts += c->npts;
        mob += c->n_mobile;
    }
    b->total_pts = pts;
    b->n_mobile = mob;
    b->total_bins = bins;
    b->flat = flat;
    b->walls = walls;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel_any(b), BT, 0);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorCooperativeLaunchTooLarge;
    b->sms = sms;
    b->max_blocks = sms * per_sm;
    // untuned: the occupancy bound's blocks per SM (or what fits)
    b->blocks = std::min(b->max_blocks, sms * (b->prec == LB_F64 ? min_blocks<double>() : min_blocks<float>()));
    // the work queue: every member's collide chunks, member after member,
    // then every member's point items
    std::vector<int> nchunk(n), skind, smember;
    std::vector<long long> sbegin;
    if (e == cudaSuccess) {
        long long units = 0;  // windows or 4-tile groups of all members
        for (int i = 0; i < n; ++i) {
            const Geom& g = ctxs[i]->geom;
            units += flat ? (g.V + 31) / 32 : (long long)work[i].groups_x * work[i].groups_y * g.nz;
        }
        const double ideal = (double)units / ((double)CHUNKS_PER_BLOCK * (double)std::max(1, b->max_blocks));
        int chunk = CHUNK_MIN;
        while (chunk < CHUNK_MAX && (double)chunk * 1.41421356 < ideal) chunk *= 2;  // nearest power of two
        b->chunk = chunk;
        long long items = 0;
        for (int i = 0; i < n; ++i) {
            const Geom& g = ctxs[i]->geom;
            const long long u = flat ? (g.V + 31) / 32 : (long long)work[i].groups_x * work[i].groups_y * g.nz;
            nchunk[i] = (int)((u + b->chunk - 1) / b->chunk);
            sbegin.push_back(items);
            smember.push_back(i);
            skind.push_back(0);
            items += nchunk[i];
        }
        for (int i = 0; i < n; ++i) {
            const long long np = (ctxs[i]->npts + NPB - 1) / NPB;
            if (np == 0) continue;
            sbegin.push_back(items);
            smember.push_back(i);
            skind.push_back(1);
            items += np;
        }
        b->total_items = items;
        b->nseg = (int)sbegin.size();
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_err, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&b->h_err, sizeof(int), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ent, sizeof(Entry) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_pbegin, sizeof(long long) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_work, sizeof(Work) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sbegin, sizeof(long long) * (size_t)b->nseg);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_smember, sizeof(int) * (size_t)b->nseg);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_skind, sizeof(int) * (size_t)b->nseg);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_nchunk, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_done, sizeof(unsigned) * n);
    if (e == cudaSuccess) e = cudaMemset(b->d_done, 0, sizeof(unsigned) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ctl, sizeof(BatchCtl));
    if (e == cudaSuccess && pts > 0)
        e = cudaMalloc(&b->d_st, lbk::arith_bytes(b->prec) * ST_W * (size_t)pts);
    if (e == cudaSuccess && pts > 0) e = cudaMalloc(&b->d_order, sizeof(int) * (size_t)pts);
    if (e == cudaSuccess && pts > 0) e = cudaMalloc(&b->d_sort, sizeof(int) * ((size_t)(3 * bins + 1) + (size_t)pts));
    if (e == cudaSuccess && pts > 0) {
        std::vector<int> pent((size_t)pts);
        for (int i = 0; i < n; ++i)
            for (long long q = pbegin[i]; q < pbegin[i] + ctxs[i]->npts; ++q) pent[(size_t)q] = i;
        e = cudaMalloc(&b->d_pent, sizeof(int) * (size_t)pts);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_pent, pent.data(), sizeof(int) * (size_t)pts, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
        BatchCtl ctl = {};
        ctl.since_sort = SORT_EVERY;  // the first step sorts
        ctl.init = 1;
        ctl.limit = DEFAULT_WAIT;
        e = cudaMemcpy(b->d_ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(b->d_ent, ent.data(), sizeof(Entry) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_pbegin, pbegin.data(), sizeof(long long) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_work, work.data(), sizeof(Work) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_sbegin, sbegin.data(), sizeof(long long) * (size_t)b->nseg, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_smember, smember.data(), sizeof(int) * (size_t)b->nseg, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_skind, skind.data(), sizeof(int) * (size_t)b->nseg, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_nchunk, nchunk.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        lb_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA;
    }
    *b->h_err = 0;
    *out = b;
    return LB_OK;
}

void lb_batch_destroy(lb_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph_ready) cudaGraphExecDestroy(b->graph2);
    cudaFree(b->d_ent);
    cudaFree(b->d_pbegin);
    cudaFree(b->d_work);
    cudaFree(b->d_sbegin);
    cudaFree(b->d_smember);
    cudaFree(b->d_skind);
    cudaFree(b->d_nchunk);
    cudaFree(b->d_done);
    cudaFree(b->d_ctl);
    cudaFree(b->d_st);
    cudaFree(b->d_pent);
    cudaFree(b->d_order);
    cudaFree(b->d_sort);
    if (b->h_err) cudaFreeHost(b->h_err);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->ev_err) cudaEventDestroy(b->ev_err);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char* lb_batch_last_error(const lb_batch* b) { return b ? b->err.c_str() : ""; }

lb_status lb_batch_set_wait_limit(lb_batch* b, long long polls) {
    if (!b) return LB_ERR_ARG;
    if (polls < 0) return bfail(b, LB_ERR_ARG, "lb_batch_set_wait_limit: polls < 0");
    LB_BCUDA(set_ctl(b, offsetof(BatchCtl, limit), &polls, sizeof(polls)), "wait limit");
    LB_BCUDA(cudaStreamSynchronize(b->stream), "stream synchronize");
    return LB_OK;
}

lb_status lb_batch_synchronize(lb_batch* b) {
    if (!b) return LB_ERR_ARG;
    LB_BCUDA(cudaStreamSynchronize(b->stream), "stream synchronize");
    if (b->err_pending) {
        b->err_pending = false;
        if (*b->h_err) {
            // a barrier wait ran out: the step's work is incomplete; reset the
            // barrier state so that later launches start clean
            *b->h_err = 0;
            LB_BCUDA(reset_sync_state(b), "barrier and queue reset");
            return bfail(b, LB_ERR_TIMEOUT, "lb_batch: a wait ran out; the last steps are incomplete");
        }
    }
    return LB_OK;
}

lb_status lb_batch_tune(lb_batch* b, int* blocks_out) {
    if (!b) return LB_ERR_ARG;
    // Whole trial steps are timed (the persistent kernel does every phase),
    // since the best grid depends on all of them.  A trial does not advance
    // the batch: the parity is not flipped, so every trial reads the same
    // current population buffers and writes the spare ones; the positions,
    // the rounding counter and the sort counter the trials move are saved
    // first and put back after the last trial, and the force fields the
    // trials spread are cleared (the next step spreads anew).
    for (lb_ctx* c : b->ctx) LB_BCUDA(cudaStreamSynchronize(c->stream), "member stream");
    LB_BCUDA(cudaStreamSynchronize(b->stream), "batch stream");
    double* saved_pos = nullptr;
    if (b->total_pts > 0) LB_BCUDA(cudaMalloc(&saved_pos, sizeof(double) * 3 * (size_t)b->total_pts), "tuner scratch");
    BatchCtl saved_ctl;
    cudaError_t err = cudaMemcpy(&saved_ctl, b->d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost);
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
        return cudaSuccess;
    };
    if (err == cudaSuccess) err = copy_positions(true);
    // trials start from cleared fields (the first trial spreads)
    if (err == cudaSuccess) err = clear_member_fields(b);
    if (err == cudaSuccess) {
        const int one = 1;
        err = set_ctl(b, offsetof(BatchCtl, init), &one, sizeof(one));
    }
    int best = b->blocks;
    float best_ms = 1e30f;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (err == cudaSuccess) err = cudaEventCreate(&t0);
    if (err == cudaSuccess) err = cudaEventCreate(&t1);
    // candidates: persistent grids of 2 to 8 blocks per SM (as many as fit)
    const int per_sm[] = {2, 4, 6, 8};
    for (int ci = 0; ci < 4 && err == cudaSuccess; ++ci) {
        const int blocks = std::min(b->max_blocks, b->sms * per_sm[ci]);
        err = launch_step(b, b->parity, blocks);  // warm
        if (err == cudaSuccess) err = cudaEventRecord(t0, b->stream);
        for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = launch_step(b, b->parity, blocks);
        if (err == cudaSuccess) err = cudaEventRecord(t1, b->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, t0, t1);
        if (err == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = blocks;
        }
        b->launches += 4;
    }
    // put the state back: positions, counters, cleared fields
    if (err == cudaSuccess) err = copy_positions(false);
    if (err == cudaSuccess) err = clear_member_fields(b);
    int timed_out = 0;
    if (err == cudaSuccess) err = cudaStreamSynchronize(b->stream);
    if (err == cudaSuccess) err = cudaMemcpy(&timed_out, &b->d_ctl->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (err == cudaSuccess) {
        saved_ctl.init = 1;
        saved_ctl.count = 0;
        saved_ctl.err = 0;
        saved_ctl.next = 0;
        saved_ctl.exits = 0;
        err = cudaMemcpy(b->d_ctl, &saved_ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice);
    }
    if (err == cudaSuccess) err = cudaMemset(b->d_done, 0, sizeof(unsigned) * (size_t)b->n);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(saved_pos);
    if (err != cudaSuccess) return bfail(b, LB_ERR_CUDA, std::string("lb_batch_tune: ") + cudaGetErrorString(err));
    if (timed_out) return bfail(b, LB_ERR_TIMEOUT, "lb_batch_tune: a wait ran out");
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
    }
    // The force fields: every member with points holds the forces at its
    // current positions (the last batch step spread them, or a query did),
    // or none does and the first step spreads.  A mixture is cleared.
    bool all_ready = true, any_ready = false;
    for (lb_ctx* c : b->ctx) {
        if (c->npts == 0) continue;
        all_ready = all_ready && c->field_ready;
        any_ready = any_ready || c->field_ready;
    }
    if (!all_ready) {
        if (any_ready) LB_BCUDA(clear_member_fields(b), "clear force field");
        const int one = 1;
        LB_BCUDA(set_ctl(b, offsetof(BatchCtl, init), &one, sizeof(one)), "spread flag");
    }
    if (!b->graph_ready && !b->graph_failed && nsteps >= 2) {
        // two cooperative launches captured as a graph; if the capture or
        // the instantiation is refused, the steps are launched one by one
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = launch_step(b, 0, b->blocks);
            if (e1 == cudaSuccess) e1 = launch_step(b, 1, b->blocks);
            e = cudaStreamEndCapture(b->stream, &g);
            if (e == cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph2, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess) b->graph_ready = true;
        else {
            cudaGetLastError();
            b->graph_failed = true;
        }
    }
    // The graph holds two steps starting at parity 0: a batch at odd parity
    // takes one plain step first.
    int done = 0;
    while (done < nsteps) {
        if (b->graph_ready && b->parity == 0 && nsteps - done >= 2) {
            LB_BCUDA(cudaGraphLaunch(b->graph2, b->stream), "graph launch");
            done += 2;
        } else {
            LB_BCUDA(launch_step(b, b->parity, b->blocks), "batched step");
            b->parity ^= 1;
            done += 1;
        }
    }
    b->launches += nsteps;
    for (lb_ctx* c : b->ctx) {
        c->cur ^= (nsteps & 1);
        c->field_ready = c->npts > 0;  // the last point phase spread the forces at the new positions
        c->stencil_ready = false;      // the member's own stencil rows and order are stale
        c->order_stale = true;
    }
    LB_BCUDA(cudaMemcpyAsync(b->h_err, &b->d_ctl->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream), "status copy");
    b->err_pending = true;
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
