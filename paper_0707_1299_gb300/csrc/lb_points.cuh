// lb_points.cuh -- per-point helpers of the colloid kernels (update,
// stencil rows), shared by the single-lattice and the batched kernels.
#pragma once

#include <type_traits>

#include "lb_device.cuh"

namespace lbk {

// The stencil row of a point (Sec. III, Eq. deltadef): the 12 Peskin
// weights phi(b + i - X) (i = 0..3, per axis) and the 3 base nodes b.  In
// FP64 every weight's offset is formed in FP64 (write_stencil); for the
// float formats the offset of the first node, b - X in (-2, -1], is
// rounded to float once and the others are r0 + i, which float holds
// exactly (each stays a multiple of r0's unit in the last place with
// magnitude at most 2): three FP64 operations an axis instead of nine.
template <typename T>
__device__ __forceinline__ void stencil_row(T* __restrict__ row, double X, double Y, double Z) {
    if constexpr (std::is_same<T, double>::value) {
        write_stencil<double>(row, X, Y, Z);
    } else {
        const double P[3] = {X, Y, Z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int b = stencil_base(P[a]);
            const float r0 = (float)((double)b - P[a]);
#pragma unroll
            for (int i = 0; i < 4; ++i) row[4 * a + i] = peskin_phi(r0 + (float)i);
            row[12 + a] = int_bits(b, T(0));
        }
        row[15] = T(0);
    }
}

// 1 / x by two Newton-Raphson steps from the float reciprocal (relative
// error 2^-23 -> 2^-46 -> within about one unit in the last place of the
// FP64 1/x, not always its correct rounding), four FP64 operations in place
// of a division; x outside the float range takes the division.
__device__ __forceinline__ double recip_fp64(double x) {
    const double ax = fabs(x);
    if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
    double r = (double)__frcp_rn((float)x);
    r = r * fma(-x, r, 2.0);
    return r * fma(-x, r, 2.0);
}

}  // namespace lbk

namespace lbk {

// ---------------------------------------------------------- point phase
// Everything the point kernels need of the lattice that holds a point: its
// geometry and fields, the point arrays and the colloid-update constants.
template <typename T>
struct PointView {
    Geom g;
    T* floc;
    flag_t* flags;
    const T* vel;
    double* pos;
    const double* force;
    const double* radius;
    const int* mobile;
    double inv_aL, inv_6pi_eta;
    int s;  // index of the point in its lattice's arrays
};

// The interpolation and the spreading take four points per warp pass:
// lanes 8u .. 8u + 7 serve point u of the pass, lane l of the eight holds
// the stencil nodes (i, j, k) with i = l % 4, j in {l / 4, l / 4 + 2} and
// all four k -- 8 nodes, 24 independent loads (or reductions) a lane, so
// that a warp keeps many memory operations in flight.  The eight lanes read
// the point's stencil row (elements l and 8 + l) and exchange its weights by
// shuffles within their group of eight.
template <typename T>
struct StencilPartT {
    int x, y0, y1;       // the lane's wrapped x node and its two y nodes
    int zk[4];           // the four z nodes
    T wxy0, wxy1;        // phi_x(i) phi_y(j), for the two j
    T wz[4];
};

template <typename T>
__device__ __forceinline__ StencilPartT<T> stencil_part(const Geom& g, const T* __restrict__ row, unsigned gmask,
                                                        int l) {
    const T e0 = row[l], e1 = row[8 + l];
    StencilPartT<T> p;
    const int i = l & 3, j0 = l >> 2;
    const T wx = __shfl_sync(gmask, e0, i, 8);
    const T wy0 = __shfl_sync(gmask, e0, 4 + j0, 8), wy1 = __shfl_sync(gmask, e0, 6 + j0, 8);
#pragma unroll
    for (int k = 0; k < 4; ++k) p.wz[k] = __shfl_sync(gmask, e1, k, 8);
    const int bx = bits_int(__shfl_sync(gmask, e1, 4, 8)), by = bits_int(__shfl_sync(gmask, e1, 5, 8)),
              bz = bits_int(__shfl_sync(gmask, e1, 6, 8));
    p.wxy0 = wx * wy0;
    p.wxy1 = wx * wy1;
    p.x = wrap_node(bx + i, g.nx);
    p.y0 = wrap_node(by + j0, g.ny);
    p.y1 = wrap_node(by + j0 + 2, g.ny);
#pragma unroll
    for (int k = 0; k < 4; ++k) p.zk[k] = wrap_node(bz + k, g.nz);
    return p;
}

// The lane's share of v(R) = sum over the 64 stencil nodes of phi phi phi v
// (Sec. IV) from the velocity the collide wrote (v = 0 on solid nodes).
template <typename T, bool WALLS>
__device__ __forceinline__ void interp_part(const PointView<T>& P, const StencilPartT<T>& sp, T acc[3]) {
    const unsigned nx = (unsigned)P.g.nx, ny = (unsigned)P.g.ny;
    acc[0] = acc[1] = acc[2] = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (WALLS && is_solid(P.g, sp.zk[k])) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const T w = (h ? sp.wxy1 : sp.wxy0) * sp.wz[k];
            const unsigned site = ((unsigned)sp.zk[k] * ny + (unsigned)(h ? sp.y1 : sp.y0)) * nx + (unsigned)sp.x;
            T vx, vy, vz;
            field_ld(P.vel, site, vx, vy, vz);
            acc[0] += w * vx;
            acc[1] += w * vy;
            acc[2] += w * vz;
        }
    }
}

// The lane's share of F delta^P(x - R) added to the force field at the
// stencil nodes (Sec. III, Eq. deltadef), flagging their 8-site groups.
template <typename T, bool WALLS>
__device__ __forceinline__ void spread_part(const PointView<T>& P, const StencilPartT<T>& sp, int l) {
    const T F0 = (T)P.force[3 * P.s], F1 = (T)P.force[3 * P.s + 1], F2 = (T)P.force[3 * P.s + 2];
    const unsigned nx = (unsigned)P.g.nx, ny = (unsigned)P.g.ny;
    const bool marker = (l & 3) == 0 || (sp.x & (GROUP_X - 1)) == 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (WALLS && is_solid(P.g, sp.zk[k])) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const T w = (h ? sp.wxy1 : sp.wxy0) * sp.wz[k];
            const unsigned rw = (unsigned)sp.zk[k] * ny + (unsigned)(h ? sp.y1 : sp.y0);
            const unsigned site = rw * nx + (unsigned)sp.x;
            field_add(P.floc, site, F0 * w, F1 * w, F2 * w);
            if (marker) P.flags[rw * (unsigned)P.g.ntx * (TILE_X / GROUP_X) + (unsigned)sp.x / GROUP_X] = 1;
        }
    }
}

// Colloid update of one point by one thread (Sec. IV, forward Euler, unit
// time step): a mobile point moves by
//   R <- R + v(R) + F (1/a - 1/a_L) / (6 pi eta)          (Eq. a_Ldefn)
// plus, with a network output y, y |F| / (6 pi eta a); wrapped
// periodically.  Returns the new position (the old one for a fixed point).
__device__ __forceinline__ double wrap_step_pos(double r, int n) {
    const double L = (double)n;
    if (r < 0.0) r += L;
    else if (r >= L) r -= L;
    if (!(r >= 0.0 && r < L)) {  // moved by a period or more
        r = r - L * floor(r / L);
        if (r >= L || r < 0.0) r = 0.0;
    }
    return r;
}

template <typename T>
__device__ __forceinline__ void update_point(const PointView<T>& P, const double v[3], const float* y, double out[3]) {
    const int s = P.s;
    out[0] = P.pos[3 * s];
    out[1] = P.pos[3 * s + 1];
    out[2] = P.pos[3 * s + 2];
    if (!P.mobile[s]) return;
    const int nn[3] = {P.g.nx, P.g.ny, P.g.nz};
    const double ia = recip_fp64(P.radius[s]);
    const double c = (ia - P.inv_aL) * P.inv_6pi_eta;
    double v0 = 0.0;
    if (y) {
        const double f0 = P.force[3 * s], f1 = P.force[3 * s + 1], f2 = P.force[3 * s + 2];
        v0 = sqrt(f0 * f0 + f1 * f1 + f2 * f2) * P.inv_6pi_eta * ia;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double r = out[a] + v[a] + P.force[3 * s + a] * c;
        if (y) r += (double)y[3 * s + a] * v0;
        out[a] = wrap_step_pos(r, nn[a]);
        P.pos[3 * s + a] = out[a];
    }
}

// The spread of a block's n points staged in shared memory (the variant
// the shared-memory pre-reduction design calls for): when the stencils of
// the block's points fit in a box of at most SHARED_NODES nodes, every
// contribution is added into a shared tile of that box first (shared-memory
// atomics), and each tile node that received force is added to the field
// with one global atomic per component -- stencils that overlap then cost
// one global reduction per node instead of one per stencil.  The groups'
// flags are set as in the direct spread.  bases[t] holds the stencil base
// of point t (as doubles); tile holds 3 SHARED_NODES elements.  Returns
// false, having done nothing, when the box does not fit (the caller then
// spreads directly).  All points of the block belong to one lattice.
constexpr int SHARED_NODES_BYTES = 40 * 1024;  // with the block's static shared memory, within the 48 KiB a launch gets without opting in
template <typename T, bool WALLS, int NP, typename Src>
__device__ __forceinline__ bool spread_block_shared(const Src& src, int n, long long gk, const T* __restrict__ st,
                                                    double (*bases)[3], T* tile, int l, unsigned gmask) {
    constexpr int MAXN = SHARED_NODES_BYTES / (3 * (int)sizeof(T));
    __shared__ int box[7];  // lo x, y, z; extent x, y, z; fits
    if (threadIdx.x == 0) {
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = (int)bases[0][a];
            hi[a] = lo[a];
        }
        for (int t = 1; t < n; ++t)
            for (int a = 0; a < 3; ++a) {
                lo[a] = min(lo[a], (int)bases[t][a]);
                hi[a] = max(hi[a], (int)bases[t][a]);
            }
        long long vol = 1;
        for (int a = 0; a < 3; ++a) {
            box[a] = lo[a];
            box[3 + a] = hi[a] - lo[a] + 4;
            vol *= box[3 + a];
        }
        box[6] = vol <= MAXN;
    }
    __syncthreads();
    if (!box[6]) return false;  // uniform per block
    const int ex = box[3], ey = box[4], ez = box[5];
    const int vol = ex * ey * ez;
    for (int q = threadIdx.x; q < 3 * vol; q += blockDim.x) tile[q] = T(0);
    __syncthreads();
    if (gk >= 0) {  // eight lanes a point, as spread_part, into the tile
        const PointView<T> P = src.view(gk);
        const T* row = st + gk * ST_W;
        const T e0 = row[l], e1 = row[8 + l];
        const int i = l & 3, j0 = l >> 2;
        const T wx = __shfl_sync(gmask, e0, i, 8);
        const T wy[2] = {__shfl_sync(gmask, e0, 4 + j0, 8), __shfl_sync(gmask, e0, 6 + j0, 8)};
        T wz[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) wz[k] = __shfl_sync(gmask, e1, k, 8);
        const int bx = bits_int(__shfl_sync(gmask, e1, 4, 8)), by = bits_int(__shfl_sync(gmask, e1, 5, 8)),
                  bz = bits_int(__shfl_sync(gmask, e1, 6, 8));
        const T F0 = (T)P.force[3 * P.s], F1 = (T)P.force[3 * P.s + 1], F2 = (T)P.force[3 * P.s + 2];
        const int xw = wrap_node(bx + i, P.g.nx);
        const bool marker = i == 0 || (xw & (GROUP_X - 1)) == 0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = j0 + 2 * h;
                const T w = wx * wy[h] * wz[k];
                const int q = ((bz + k - box[2]) * ey + (by + j - box[1])) * ex + (bx + i - box[0]);
                atomicAdd(&tile[3 * q], F0 * w);
                atomicAdd(&tile[3 * q + 1], F1 * w);
                atomicAdd(&tile[3 * q + 2], F2 * w);
                const int zw = wrap_node(bz + k, P.g.nz);
                if (marker && !(WALLS && is_solid(P.g, zw))) {
                    const unsigned rw = (unsigned)zw * (unsigned)P.g.ny + (unsigned)wrap_node(by + j, P.g.ny);
                    P.flags[rw * (unsigned)P.g.ntx * (TILE_X / GROUP_X) + (unsigned)xw / GROUP_X] = 1;
                }
            }
    }
    __syncthreads();
    const PointView<T> P = src.view(0);  // the lattice of every point of the block
    for (int q = threadIdx.x; q < vol; q += blockDim.x) {
        const T f0 = tile[3 * q], f1 = tile[3 * q + 1], f2 = tile[3 * q + 2];
        if (f0 == T(0) && f1 == T(0) && f2 == T(0)) continue;
        const int x = wrap_node(box[0] + q % ex, P.g.nx), y = wrap_node(box[1] + (q / ex) % ey, P.g.ny),
                  z = wrap_node(box[2] + q / (ex * ey), P.g.nz);
        if (WALLS && is_solid(P.g, z)) continue;
        const unsigned site = ((unsigned)z * (unsigned)P.g.ny + (unsigned)y) * (unsigned)P.g.nx + (unsigned)x;
        field_add(P.floc, site, f0, f1, f2);
    }
    return true;
}

// The point phase of one block of NW warps over up to 4 NW consecutive
// slots of the work order (slot0 ..; point of slot q = order[q], or q
// itself without an order), in three parts separated by block barriers:
//   1. every colloid's velocity is interpolated at its current position,
//      four points a warp (eight lanes a point), the sums kept in shared
//      memory (vsh, 4 NW x 3 doubles);
//   2. thread t < 4 NW moves point t (FP64, a lane a point: the SM's FP64
//      unit costs the same for a warp instruction with one lane active as
//      with 32) and writes the stencil row of its new position;
//   3. every point's force is spread at its new position for the next
//      step, four points a warp.
// With INTERP false only the stencil rows and the spread at the current
// positions run (a first spread).  src.view(gp) gives a point's PointView,
// src.y(gp) its network output rows (or null).  Every thread of the block
// must call it (it holds block barriers).
template <typename T, bool WALLS, bool INTERP, int NW, typename Src, bool SHARED = false>
__device__ __forceinline__ void point_block(const Src& src, long long slot0, long long total,
                                            const int* __restrict__ order, T* __restrict__ st,
                                            double (*vsh)[3], T* tile = nullptr) {
    constexpr int NP = 4 * NW;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = (int)min((long long)NP, total - slot0);
    const int u = lane >> 3, l = lane & 7;
    const unsigned gmask = 0xFFu << (8 * u);
    const int k = 4 * warp + u;  // this group of eight's point in parts 1 and 3
    const long long gk = k < n ? (long long)(order ? order[slot0 + k] : slot0 + k) : -1LL;
    if (INTERP) {
        T acc[3] = {T(0), T(0), T(0)};
        if (gk >= 0) {  // uniform per group of eight
            const PointView<T> P = src.view(gk);
            // the stencil row is loaded beside the mobile flag, not after it
            const int mob = P.mobile[P.s];
            const StencilPartT<T> sp = stencil_part<T>(P.g, st + gk * ST_W, gmask, l);
            if (mob) interp_part<T, WALLS>(P, sp, acc);
        }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1)
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], off);
        if (l == 0 && gk >= 0)
#pragma unroll
            for (int a = 0; a < 3; ++a) vsh[k][a] = (double)acc[a];
    }
    __syncthreads();
    if ((int)threadIdx.x < n) {
        const int t = threadIdx.x;
        const long long gp = order ? order[slot0 + t] : slot0 + t;
        const PointView<T> P = src.view(gp);
        double R[3];
        if (INTERP) {
            const double v[3] = {vsh[t][0], vsh[t][1], vsh[t][2]};
            update_point<T>(P, v, src.y(gp), R);
        } else {
            R[0] = P.pos[3 * P.s];
            R[1] = P.pos[3 * P.s + 1];
            R[2] = P.pos[3 * P.s + 2];
        }
        stencil_row<T>(st + gp * ST_W, R[0], R[1], R[2]);
        if (SHARED)
#pragma unroll
            for (int a = 0; a < 3; ++a) vsh[t][a] = floor(R[a]) - 1.0;  // stencil base, for the block's box
    }
    __syncthreads();
    if (SHARED && n > 0 && spread_block_shared<T, WALLS, NP>(src, n, gk, st, vsh, tile, l, gmask)) return;
    if (gk >= 0) {
        const PointView<T> P = src.view(gk);
        const StencilPartT<T> sp = stencil_part<T>(P.g, st + gk * ST_W, gmask, l);
        spread_part<T, WALLS>(P, sp, l);
    }
}

}  // namespace lbk
