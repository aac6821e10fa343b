// lb_kernels.cu -- sm_103a kernels of the forced D3Q19 MRT lattice
// Boltzmann method with singular point forces, and their launchers.
//
//   (the collide kernels are in lb_collide.cu: they read the localised
//   force only in the 8-site groups flagged by the spread and, for
//   lattices with colloids, write the fluid velocity there and zero the
//   consumed force and flags)
//   k_points    the point phase after the collide: colloid velocity
//               interpolated with the same kernel from the velocity the
//               collide wrote (Sec. IV), the update
//               R += v(R) + F (1/a - 1/a_L) / (6 pi eta) (Eq. a_Ldefn), and
//               the spread at the new positions for the next step
//               (regularised point forces, Sec. III, Eq. deltadef: the 12
//               one-dimensional weights evaluated once and shuffled,
//               atomic accumulation into the field); without the
//               interpolation, the first spread of a set of points.
//   k_gather    velocity at arbitrary query points, each stencil node
//               rebuilt from its pulled populations.
//   k_moments   rho, u fields and FP64 totals (Eq. macrovariables2).
#include <math.h>

#include <algorithm>

#include "../../include/lb.h"
#include "lb_internal.h"
#include "lb_points.cuh"

namespace lbk {


size_t storage_bytes(int prec) {
    switch (prec) {
        case LB_F64: return 8;
        case LB_F32: return 4;
        default: return 2;
    }
}
size_t arith_bytes(int prec) { return prec == LB_F64 ? 8 : 4; }

double n_fluid(const lb_ctx* c) {
    long long nfluid = c->geom.V;
    const long long plane = (long long)c->geom.nx * c->geom.ny;
    if (c->geom.wall_lo >= 0) nfluid -= plane;
    if (c->geom.wall_hi >= 0 && c->geom.wall_hi != c->geom.wall_lo) nfluid -= plane;
    return (double)nfluid;
}

// Uniform force density on fluid sites: g plus the counter-force
// -sum F / V_fluid (evaluated on the host in FP64, passed in the arithmetic type).
template <typename T>
UForce<T> uniform_force(const lb_ctx* c) {  // instantiated for float and double below
    UForce<T> u;
    const double nf = n_fluid(c);
    for (int a = 0; a < 3; ++a) {
        double F = c->g[a];
        if (c->counter && c->npts > 0 && nf > 0) F -= c->fsum_host[a] / nf;
        u.F[a] = (T)F;
    }
    return u;
}

template UForce<float> uniform_force<float>(const lb_ctx*);
template UForce<double> uniform_force<double>(const lb_ctx*);

// Compact list of the flagged tiles (at most cap written; *count gets the
// total).  One warp per 32 flags.
__global__ void k_list_tiles(const flag_t* __restrict__ flags, long long ntiles, unsigned* __restrict__ list,
                             unsigned cap, unsigned* __restrict__ count) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool mine = t < ntiles && ((const unsigned*)flags)[t] != 0u;
    const unsigned m = __ballot_sync(0xffffffffu, mine);
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (lane == 0 && m) base = atomicAdd(count, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (mine) {
        const unsigned idx = base + (unsigned)__popc(m & ((1u << lane) - 1u));
        if (idx < cap) list[idx] = (unsigned)t;
    }
}


// Position wrapped into [0, n).
__device__ __forceinline__ double wrap_pos(double r, int n) {
    const double L = (double)n;
    r = r - L * floor(r / L);
    if (r >= L || r < 0.0) r = 0.0;
    return r;
}


// Stencil rows of n points.
template <typename T>
__global__ void k_stencil(int n, const double* __restrict__ pos, T* __restrict__ st) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    stencil_row<T>(st + (size_t)t * ST_W, pos[3 * t], pos[3 * t + 1], pos[3 * t + 2]);
}

// ------------------------------------------------------------- k_points
// The point phase of a lattice with colloids, after its collide: a block of
// 2 warps per 8 points in cell order (point_block): every colloid's
// velocity is interpolated from the velocity field the collide wrote, every
// point moves (Sec. IV update, with the network output y when a correction
// is attached) and its stencil row is rewritten, and the forces are spread
// at the new positions for the next step.
template <typename T>
struct LatticePoints {
    PointView<T> v;
    const float* yc;
    __device__ __forceinline__ PointView<T> view(long long gp) const {
        PointView<T> p = v;
        p.s = (int)gp;
        return p;
    }
    __device__ __forceinline__ const float* y(long long) const { return yc; }
};

// warps of a k_points block (8 points): measured on GB300 against 8 and 4
// warps (32 and 16 points), the small block is 7 % (1e5 colloids in 512^3)
// and 13 % (2e5 in 256^3) faster -- the phase waits on memory, and fewer
// warps a block barrier hold fewer warps idle
constexpr int PT_WARPS = 2;

// With INTERP false the kernel only writes the stencil rows at the current
// positions and spreads there: the first spread of a set of points.
template <typename T, bool WALLS, bool SHARED, bool INTERP = true>
__global__ void __launch_bounds__(PT_WARPS * 32) k_points(const LatticePoints<T> src, long long total,
                                                          const int* __restrict__ order, T* __restrict__ st) {
    __shared__ double vsh[4 * PT_WARPS][3];
    extern __shared__ __align__(16) unsigned char pt_tile[];
    point_block<T, WALLS, INTERP, PT_WARPS, LatticePoints<T>, SHARED>(src, (long long)blockIdx.x * (4 * PT_WARPS),
                                                                      total, order, st, vsh, (T*)pt_tile);
}

// ------------------------------------------------------------- k_gather
// v at n query points (Sec. IV interpolation), one warp per point, two
// stencil nodes per lane, each node's v rebuilt from its pulled populations
// and the force at time n (Eq. macrovariables2).
template <typename S, bool WALLS>
__global__ void __launch_bounds__(128)
k_gather(const Pops<S> src, const typename Store<S>::T* __restrict__ floc, Geom g, UForce<typename Store<S>::T> fu,
         float inv_scale, int n, const double* __restrict__ qpos, double* __restrict__ vout) {
    using T = typename Store<S>::T;
    const int s = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (s >= n) return;
    const int lane = threadIdx.x & 31;
    const double* P = qpos + 3 * s;
    const double X = wrap_pos(P[0], g.nx), Y = wrap_pos(P[1], g.ny), Z = wrap_pos(P[2], g.nz);
    const StencilLane<T> st = stencil_lane<T>(X, Y, Z, lane);
    const unsigned FULL = 0xffffffffu;
    const int bx = __shfl_sync(FULL, st.base, 0), by = __shfl_sync(FULL, st.base, 4), bz = __shfl_sync(FULL, st.base, 8);
    T acc[3] = {T(0), T(0), T(0)};
    for (int h = 0; h < 2; ++h) {
        const int node = lane + 32 * h;
        const int i = node & 3, j = (node >> 2) & 3, k = node >> 4;
        const T w = __shfl_sync(FULL, st.phi, i) * __shfl_sync(FULL, st.phi, 4 + j) * __shfl_sync(FULL, st.phi, 8 + k);
        const int x = wrap_node(bx + i, g.nx), y = wrap_node(by + j, g.ny), z = wrap_node(bz + k, g.nz);
        if (WALLS && is_solid(g, z)) continue;  // v = 0 on solid nodes
        const Nbr nb = neighbours(g, x, y, z);
        const unsigned site = nb.c + nb.x;
        T f[NQ];
        pull19<S, WALLS>(src, nb, f);
        unscale19<S>(f, inv_scale);
        T lx, ly, lz;
        field_ld(floc, site, lx, ly, lz);
        const T Fx = fu.F[0] + lx, Fy = fu.F[1] + ly, Fz = fu.F[2] + lz;
        T drho, vx, vy, vz;
        macro19<T, Store<S>::kCompensate>(f, Fx, Fy, Fz, drho, vx, vy, vz);
        acc[0] += w * vx;
        acc[1] += w * vy;
        acc[2] += w * vz;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        for (int a = 0; a < 3; ++a) acc[a] += __shfl_xor_sync(FULL, acc[a], off);
    if (lane == 0)
        for (int a = 0; a < 3; ++a) vout[3 * s + a] = (double)acc[a];
}

// ------------------------------------------------------------ k_moments
// Grid-stride over tiles; each block writes 4 FP64 partial sums
// (rho, rho u) in a fixed order, so the totals are deterministic.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int w = tid >> 5, lane = tid & 31;
    const int nw = (int)(blockDim.x * blockDim.y) >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (tid == 0)
        for (int i = 0; i < nw; ++i) t += sh[i];
    return t;  // valid in thread 0
}

template <typename S, bool WALLS>
__global__ void __launch_bounds__(CS_THREADS)
k_moments(const Pops<S> src, const typename Store<S>::T* __restrict__ floc, Geom g, UForce<typename Store<S>::T> fu,
          float inv_scale, double* __restrict__ rho_out, double* __restrict__ u_out, double* __restrict__ partials) {
    using T = typename Store<S>::T;
    __shared__ double sh[CS_WARPS];
    const int y = blockIdx.y * CS_WARPS + threadIdx.y;
    const int z = blockIdx.z, lane = threadIdx.x;
    const int x = blockIdx.x * TILE_X + lane;
    const unsigned V = (unsigned)g.V;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (y < g.ny && x < g.nx) {
        const Nbr nb = neighbours(g, x, y, z);
        const unsigned site = nb.c + nb.x;
        double r = 1.0, u[3] = {0.0, 0.0, 0.0};
        if (!(WALLS && is_solid(g, z))) {
            T f[NQ];
            pull19<S, WALLS>(src, nb, f);
            unscale19<S>(f, inv_scale);
            T lx, ly, lz;
            field_ld(floc, site, lx, ly, lz);
            const T Fx = fu.F[0] + lx, Fy = fu.F[1] + ly, Fz = fu.F[2] + lz;
            T drho, vx, vy, vz;
            macro19<T, Store<S>::kCompensate>(f, Fx, Fy, Fz, drho, vx, vy, vz);
            r = 1.0 + (double)drho;
            u[0] = (double)vx;
            u[1] = (double)vy;
            u[2] = (double)vz;
            acc[0] = r;
            for (int a = 0; a < 3; ++a) acc[1 + a] = r * u[a];
        }
        if (rho_out) rho_out[site] = r;
        if (u_out)
            for (int a = 0; a < 3; ++a) u_out[(size_t)a * V + site] = u[a];
    }
    if (partials) {
        const unsigned b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        for (int a = 0; a < 4; ++a) {
            const double t = block_sum(acc[a], sh);
            if (threadIdx.x == 0 && threadIdx.y == 0) partials[4 * (size_t)b + a] = t;
        }
    }
}

__global__ void k_reduce_partials(const double* __restrict__ partials, long long nblocks, double* __restrict__ out) {
    __shared__ double sh[32];
    for (int a = 0; a < 4; ++a) {
        double v = 0.0;
        for (long long b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[4 * b + a];
        const double t = block_sum(v, sh);
        if (threadIdx.x == 0) out[a] = t;
    }
}

// U = v(R) + F (1/a - 1/a_L) / (6 pi eta): the colloid velocity of Sec. IV
// from the interpolated fluid velocity v (in place).
__global__ void k_faxen(int n, const double* __restrict__ F, const double* __restrict__ a, double inv_aL,
                        double inv_6pi_eta, double* __restrict__ U) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double c = (1.0 / a[t] - inv_aL) * inv_6pi_eta;
    for (int k = 0; k < 3; ++k) U[3 * t + k] += F[3 * t + k] * c;
}


// ---------------------------------------------------- point bookkeeping

// Expand n records of one kind into monopoles at out offset `base`
// (Sec. III: stresslet = collinear pair, rotlet = four tangential forces).
__global__ void k_expand(const double* __restrict__ pos, const double* __restrict__ F,
                         const double* __restrict__ param, int n, int kind, int base, Geom g,
                         double* __restrict__ opos, double* __restrict__ oforce, double* __restrict__ orad,
                         int* __restrict__ omob, int* __restrict__ status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double p[3], f[3];
    bool finite = true;
    for (int a = 0; a < 3; ++a) {
        p[a] = pos[3 * t + a];
        f[a] = F[3 * t + a];
        finite = finite && isfinite(p[a]) && isfinite(f[a]);
    }
    const double prm = param ? param[t] : 0.0;
    if (param) finite = finite && isfinite(prm);
    if (!finite) {
        atomicOr(status, 1);
        return;
    }
    const double nrm = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if ((kind != LB_STOKESLET && !(prm > 0.0)) || ((kind == LB_STRESSLET || kind == LB_ROTLET) && !(nrm > 0.0))) {
        atomicOr(status, 2);
        return;
    }
    const int nn[3] = {g.nx, g.ny, g.nz};
    double P[4][3], Fo[4][3];
    int m = 1;
    if (kind == LB_STOKESLET || kind == LB_COLLOID) {
        for (int a = 0; a < 3; ++a) {
            P[0][a] = p[a];
            Fo[0][a] = f[a];
        }
    } else if (kind == LB_STRESSLET) {
        m = 2;
        for (int a = 0; a < 3; ++a) {
            const double d = f[a] / nrm * (prm / 2);
            P[0][a] = p[a] + d;
            P[1][a] = p[a] - d;
            Fo[0][a] = f[a];
            Fo[1][a] = -f[a];
        }
    } else {  // rotlet
        m = 4;
        double t_hat[3] = {f[0] / nrm, f[1] / nrm, f[2] / nrm};
        int kmin = 0;
        for (int a = 1; a < 3; ++a)
            if (fabs(t_hat[a]) < fabs(t_hat[kmin])) kmin = a;
        double e1[3] = {0.0, 0.0, 0.0};
        e1[kmin] = 1.0;
        const double dot = t_hat[kmin];
        for (int a = 0; a < 3; ++a) e1[a] -= dot * t_hat[a];
        const double n1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        for (int a = 0; a < 3; ++a) e1[a] /= n1;
        const double e2[3] = {t_hat[1] * e1[2] - t_hat[2] * e1[1], t_hat[2] * e1[0] - t_hat[0] * e1[2],
                              t_hat[0] * e1[1] - t_hat[1] * e1[0]};
        const double h = prm / 2, mag = nrm / (2 * prm);
        for (int a = 0; a < 3; ++a) {
            P[0][a] = p[a] + h * e1[a];
            Fo[0][a] = mag * e2[a];
            P[1][a] = p[a] - h * e1[a];
            Fo[1][a] = -mag * e2[a];
            P[2][a] = p[a] + h * e2[a];
            Fo[2][a] = -mag * e1[a];
            P[3][a] = p[a] - h * e2[a];
            Fo[3][a] = mag * e1[a];
        }
    }
    for (int q = 0; q < m; ++q) {
        const long long o = (long long)base + (long long)t * m + q;
        for (int a = 0; a < 3; ++a) {
            opos[3 * o + a] = wrap_pos(P[q][a], nn[a]);
            oforce[3 * o + a] = Fo[q][a];
        }
        orad[o] = (kind == LB_COLLOID) ? prm : 0.0;
        omob[o] = (kind == LB_COLLOID) ? 1 : 0;
    }
}

__global__ void k_fsum(const double* __restrict__ force, int npts, double* __restrict__ out) {
    __shared__ double sh[32];
    for (int a = 0; a < 3; ++a) {
        double v = 0.0;
        for (int s = threadIdx.x; s < npts; s += blockDim.x) v += force[3 * s + a];
        const double t = block_sum(v, sh);
        if (threadIdx.x == 0) out[a] = t;
    }
}

// New positions: with pos null only the check (status set where a value
// is not finite), else the wrapped copy of values already checked, so a
// rejected update leaves every position as it was.
__global__ void k_set_positions(const double* __restrict__ in, int npts, Geom g, double* __restrict__ pos,
                                int* __restrict__ status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npts) return;
    const int nn[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a) {
        const double r = in[3 * t + a];
        if (!pos) {
            if (!isfinite(r)) atomicOr(status, 1);
        } else {
            pos[3 * t + a] = wrap_pos(r, nn[a]);
        }
    }
}

template <typename S>
__global__ void k_convert_out(const S* __restrict__ src, long long count, float inv_scale, double* __restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)Store<S>::ld(src, (unsigned)i) * (double)inv_scale;
}

template <typename S>
__global__ void k_convert_in(const double* __restrict__ in, long long count, float scale, S* __restrict__ dst,
                             unsigned seed) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
        unsigned r = rng_seed((unsigned)i, seed);
        Store<S>::st(dst, (unsigned)i, (typename Store<S>::T)(in[i] * (double)scale), rng_next(r));
    }
}

// -------------------------------------------------------------- a_L sum
// (1/a_L) = (6 pi / V) sum_{k != 0} |delta^P(k;R)|^2 / k^2 d.(1 - k^k^).d,
// Appendix A; the transform of the stencil factorises over the axes.
__global__ void k_aL(int nx, int ny, int nz, double Rx, double Ry, double Rz, double dx, double dy, double dz,
                     int iso, double* __restrict__ partials) {
    __shared__ double sh[32];
    const long long V = (long long)nx * ny * nz;
    const int nn[3] = {nx, ny, nz};
    const double R[3] = {Rx, Ry, Rz}, d[3] = {dx, dy, dz};
    double acc = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < V; t += (long long)gridDim.x * blockDim.x) {
        long long m[3] = {t % nx, (t / nx) % ny, t / ((long long)nx * ny)};
        if (m[0] == 0 && m[1] == 0 && m[2] == 0) continue;
        double k[3], d2 = 1.0;
        for (int a = 0; a < 3; ++a) {
            const long long n = nn[a];
            const long long ms = (m[a] > n / 2) ? m[a] - n : m[a];
            k[a] = 2.0 * M_PI * (double)ms / (double)n;
            const int b = (int)floor(R[a]) - 1;
            double re = 0.0, im = 0.0;
            for (int j = b; j < b + 4; ++j) {
                const double w = peskin_phi((double)j - R[a]);
                const long long ph = (((long long)ms * j) % n + n) % n;  // e^{-i 2 pi ms j / n}
                double sn, cs;
                sincospi(2.0 * (double)ph / (double)n, &sn, &cs);
                re += w * cs;
                im -= w * sn;
            }
            d2 *= re * re + im * im;
        }
        const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        double proj;
        if (iso) {
            proj = 2.0 / 3.0;
        } else {
            const double kd = k[0] * d[0] + k[1] * d[1] + k[2] * d[2];
            proj = 1.0 - kd * kd / k2;
        }
        acc += d2 / k2 * proj;
    }
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void k_sum1(const double* __restrict__ partials, int n, double* __restrict__ out) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) v += partials[b];
    const double t = block_sum(v, sh);
    if (threadIdx.x == 0) out[0] = t;
}

// ----------------------------------------------------------- cell order
// The points ordered by the 8^3 brick that holds them (a counting sort), so
// that warps next to each other in a launch work on nearby stencils: the
// spread's atomics and the interpolation's loads then find their lines in
// L2.  Only the order of the work depends on it, never a result.
constexpr int BRICK = 8;

__global__ void k_brick_count(const double* __restrict__ pos, int n, Geom g, int3 nb, int* __restrict__ count,
                              int* __restrict__ key) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int bx = min(max((int)pos[3 * t] / BRICK, 0), nb.x - 1);
    const int by = min(max((int)pos[3 * t + 1] / BRICK, 0), nb.y - 1);
    const int bz = min(max((int)pos[3 * t + 2] / BRICK, 0), nb.z - 1);
    const int b = (bz * nb.y + by) * nb.x + bx;
    key[t] = b;
    atomicAdd(&count[b], 1);
}

__global__ void k_brick_fill(int n, const int* __restrict__ key, const int* __restrict__ start,
                             int* __restrict__ cursor, int* __restrict__ order) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int b = key[t];
    order[start[b] + atomicAdd(&cursor[b], 1)] = t;
}

// ---------------------------------------------------- exclusive int scan
// Three passes: tile sums, a one-block scan of the tile sums, and the scan
// of each tile offset by its prefix.  Tiles of 2048 ints; at most 8192 tiles.
constexpr int SCAN_T = 256, SCAN_PER = 8, SCAN_TILE = SCAN_T * SCAN_PER, SCAN_MAX_TILES = 8192;

__device__ __forceinline__ int warp_inclusive_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive prefix of v over the block (blockDim.x a multiple of 32);
// *total gets the block's sum.  sh: 33 ints of shared memory.
__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)blockDim.x >> 5;
    const int inc = warp_inclusive_scan(v);
    __syncthreads();
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int x = lane < nw ? sh[lane] : 0;
        const int xi = warp_inclusive_scan(x);
        if (lane < nw) sh[lane] = xi - x;
        if (lane == 31) sh[32] = xi;
    }
    __syncthreads();
    *total = sh[32];
    return sh[w] + inc - v;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const int* __restrict__ in, long long m, int* __restrict__ bsum) {
    __shared__ int sh[33];
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    int v = 0;
#pragma unroll
    for (int r = 0; r < SCAN_PER; ++r) {
        const long long i = base + r * SCAN_T + threadIdx.x;
        if (i < m) v += in[i];
    }
    int total;
    block_exclusive_scan(v, sh, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// One block of 1024 threads: exclusive scan of the nt tile sums in place,
// the grand total in bsum[nt].
__global__ void __launch_bounds__(1024) k_scan_top(int* __restrict__ bsum, int nt) {
    __shared__ int sh[33];
    const int per = (nt + 1023) / 1024;  // at most 8
    const int b = threadIdx.x * per;
    int loc[8];
    int v = 0;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        loc[r] = (r < per && b + r < nt) ? bsum[b + r] : 0;
        v += loc[r];
    }
    int total;
    int run = block_exclusive_scan(v, sh, &total);
#pragma unroll
    for (int r = 0; r < 8; ++r)
        if (r < per && b + r < nt) {
            bsum[b + r] = run;
            run += loc[r];
        }
    if (threadIdx.x == 0) bsum[nt] = total;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_apply(const int* __restrict__ in, long long m,
                                                       const int* __restrict__ bsum, int nt, int* __restrict__ out) {
    __shared__ int sh[33];
    const long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_PER;
    int loc[SCAN_PER];
    int v = 0;
#pragma unroll
    for (int r = 0; r < SCAN_PER; ++r) {
        loc[r] = base + r < m ? in[base + r] : 0;
        v += loc[r];
    }
    int total;
    int run = block_exclusive_scan(v, sh, &total) + bsum[blockIdx.x];
#pragma unroll
    for (int r = 0; r < SCAN_PER; ++r)
        if (base + r < m) {
            out[base + r] = run;
            run += loc[r];
        }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[m] = bsum[nt];
}

size_t scan_ws_ints(long long m) { return (size_t)((m + SCAN_TILE - 1) / SCAN_TILE) + 1; }

cudaError_t scan_exclusive(const int* in, long long m, int* out, int* bsum, cudaStream_t st) {
    const long long nt = (m + SCAN_TILE - 1) / SCAN_TILE;
    if (nt > SCAN_MAX_TILES) return cudaErrorInvalidValue;
    if (nt == 0) return cudaMemsetAsync(out, 0, sizeof(int), st);
    k_scan_reduce<<<(unsigned)nt, SCAN_T, 0, st>>>(in, m, bsum);
    k_scan_top<<<1, 1024, 0, st>>>(bsum, (int)nt);
    k_scan_apply<<<(unsigned)nt, SCAN_T, 0, st>>>(in, m, bsum, (int)nt, out);
    return cudaGetLastError();
}

static int3 brick_dims(const Geom& g) {
    return make_int3((g.nx + BRICK - 1) / BRICK, (g.ny + BRICK - 1) / BRICK, (g.nz + BRICK - 1) / BRICK);
}

// Workspace of the cell-order sort, in ints: count and cursor (nb each),
// start (nb + 1), the tile sums of the scan, and one key per point.
size_t sort_ws_ints(const Geom& g, long long npts) {
    const int3 d = brick_dims(g);
    const long long nb = (long long)d.x * d.y * d.z;
    return (size_t)(3 * nb + 1) + scan_ws_ints(nb) + (size_t)npts;
}

// The flagged tiles of a field of fixed points, listed for the fix-up when
// they are few: a point flags at most 32 tiles (16 node rows, two x-tiles
// each), so with npts * 32 within the list's capacity (1/64 of all tiles,
// at least 1024) every flagged tile fits, and nothing is read back.
cudaError_t list_fixed_tiles(lb_ctx* c) {
    const unsigned cap = fixed_tile_cap(c);
    c->fix_ok = (long long)c->npts * 32 <= (long long)cap;
    if (!c->fix_ok) return cudaSuccess;
    if (!c->fix_list) {
        cudaError_t e = cudaMalloc(&c->fix_list, sizeof(unsigned) * (cap + 1));
        if (e != cudaSuccess) {
            c->fix_ok = false;
            return e;
        }
    }
    unsigned* count = c->fix_list + cap;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return e;
    k_list_tiles<<<(unsigned)((c->geom.ntiles + 255) / 256), 256, 0, c->stream>>>(c->flags, c->geom.ntiles, c->fix_list,
                                                                                 cap, count);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t ensure_velocity_field(lb_ctx* c) {
    if (c->vel || c->n_mobile == 0) return cudaSuccess;
    return cudaMalloc(&c->vel, arith_bytes(c->prec) * FIELD_W * (size_t)c->geom.V);
}

cudaError_t launch_sort_points(lb_ctx* c) {
    if (c->npts == 0) return cudaSuccess;
    const int3 d = brick_dims(c->geom);
    const long long nb = (long long)d.x * d.y * d.z;
    int* count = c->sort_ws;
    int* cursor = count + nb;
    int* start = cursor + nb;
    int* bsum = start + nb + 1;
    int* key = bsum + scan_ws_ints(nb);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * 2 * (size_t)nb, c->stream);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((c->npts + 255) / 256);
    k_brick_count<<<blocks, 256, 0, c->stream>>>(c->pos, c->npts, c->geom, d, count, key);
    e = scan_exclusive(count, nb, start, bsum, c->stream);
    if (e != cudaSuccess) return e;
    k_brick_fill<<<blocks, 256, 0, c->stream>>>(c->npts, key, start, cursor, c->order);
    c->launches += 5;
    return cudaGetLastError();
}

// ------------------------------------------------------------ launchers

// The cell order of the points, or null (their own order) for a few.
static const int* point_order(const lb_ctx* c) { return c->npts > SORT_MIN_POINTS ? c->order : nullptr; }

// The point arrays and fields of a context for the point kernels (network
// output y of the correction, or null).
template <typename T>
static LatticePoints<T> lattice_points(const lb_ctx* c, const float* y) {
    LatticePoints<T> src;
    src.v.g = c->geom;
    src.v.floc = (T*)c->floc;
    src.v.flags = c->flags;
    src.v.vel = (const T*)c->vel;
    src.v.pos = c->pos;
    src.v.force = c->force;
    src.v.radius = c->radius;
    src.v.mobile = c->mobile;
    src.v.inv_aL = isinf(c->a_L) ? 0.0 : 1.0 / c->a_L;
    src.v.inv_6pi_eta = 1.0 / (6.0 * M_PI * (c->tau_s / 3.0));
    src.v.s = 0;
    src.yc = y;
    return src;
}

template <typename T>
static cudaError_t spread_t(lb_ctx* c) {
    const LatticePoints<T> src = lattice_points<T>(c, nullptr);
    const unsigned blocks = (unsigned)((c->npts + 4 * PT_WARPS - 1) / (4 * PT_WARPS));
    const int* ord = point_order(c);
    T* st = (T*)c->stencil;
    if (has_walls(c)) k_points<T, true, false, false><<<blocks, PT_WARPS * 32, 0, c->stream>>>(src, c->npts, ord, st);
    else k_points<T, false, false, false><<<blocks, PT_WARPS * 32, 0, c->stream>>>(src, c->npts, ord, st);
    c->launches++;
    return cudaGetLastError();
}

// Stencil rows at the current positions and the spread there (Sec. III).
cudaError_t launch_spread(lb_ctx* c) {
    if (c->npts == 0) return cudaSuccess;
    return c->prec == LB_F64 ? spread_t<double>(c) : spread_t<float>(c);
}

template <typename S>
static cudaError_t gather_t(lb_ctx* c, int n, const double* qpos, double* vout) {
    using T = typename Store<S>::T;
    const UForce<T> fu = uniform_force<T>(c);
    const unsigned int blocks = (unsigned int)((n + 3) / 4);
    const Pops<S> src = pops<S>(c->f[c->cur], c->geom.V);
    if (has_walls(c))
        k_gather<S, true><<<blocks, 128, 0, c->stream>>>(src, (const T*)c->floc, c->geom, fu, c->inv_scale, n, qpos,
                                                          vout);
    else
        k_gather<S, false><<<blocks, 128, 0, c->stream>>>(src, (const T*)c->floc, c->geom, fu, c->inv_scale, n, qpos,
                                                           vout);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_gather(lb_ctx* c, int n, const double* qpos, double* vout) {
    if (n == 0) return cudaSuccess;
    switch (c->prec) {
        case LB_F64: return gather_t<double>(c, n, qpos, vout);
        case LB_F32: return gather_t<float>(c, n, qpos, vout);
        case LB_F16S: return gather_t<__half>(c, n, qpos, vout);
        default: return gather_t<__nv_bfloat16>(c, n, qpos, vout);
    }
}

template <typename T>
static cudaError_t points_t(lb_ctx* c, const float* y) {
    const LatticePoints<T> src = lattice_points<T>(c, y);
    const unsigned blocks = (unsigned)((c->npts + 4 * PT_WARPS - 1) / (4 * PT_WARPS));
    const size_t tile = SHARED_NODES_BYTES;
    const int* ord = point_order(c);
    T* st = (T*)c->stencil;
    if (c->spread_shared) {
        if (has_walls(c)) k_points<T, true, true><<<blocks, PT_WARPS * 32, tile, c->stream>>>(src, c->npts, ord, st);
        else k_points<T, false, true><<<blocks, PT_WARPS * 32, tile, c->stream>>>(src, c->npts, ord, st);
    } else {
        if (has_walls(c)) k_points<T, true, false><<<blocks, PT_WARPS * 32, 0, c->stream>>>(src, c->npts, ord, st);
        else k_points<T, false, false><<<blocks, PT_WARPS * 32, 0, c->stream>>>(src, c->npts, ord, st);
    }
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_points(lb_ctx* c, const float* y) {
    if (c->npts == 0) return cudaSuccess;
    return c->prec == LB_F64 ? points_t<double>(c, y) : points_t<float>(c, y);
}

cudaError_t launch_stencil(lb_ctx* c) {
    if (c->npts == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((c->npts + 127) / 128);
    if (c->prec == LB_F64) k_stencil<double><<<blocks, 128, 0, c->stream>>>(c->npts, c->pos, (double*)c->stencil);
    else k_stencil<float><<<blocks, 128, 0, c->stream>>>(c->npts, c->pos, (float*)c->stencil);
    c->launches++;
    return cudaGetLastError();
}

long long moment_blocks(const Geom& g) {
    const dim3 gr = site_grid(g);
    return (long long)gr.x * gr.y * gr.z;
}

template <typename S>
static cudaError_t moments_t(lb_ctx* c, double* rho, double* u, bool want_totals) {
    using T = typename Store<S>::T;
    const UForce<T> fu = uniform_force<T>(c);
    const Pops<S> src = pops<S>(c->f[c->cur], c->geom.V);
    double* part = want_totals ? c->partials : nullptr;
    if (has_walls(c))
        k_moments<S, true><<<site_grid(c->geom), site_block(), 0, c->stream>>>(src, (const T*)c->floc, c->geom, fu,
                                                                               c->inv_scale, rho, u, part);
    else
        k_moments<S, false><<<site_grid(c->geom), site_block(), 0, c->stream>>>(src, (const T*)c->floc, c->geom, fu,
                                                                                c->inv_scale, rho, u, part);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !want_totals) return e;
    k_reduce_partials<<<1, 1024, 0, c->stream>>>(c->partials, moment_blocks(c->geom), c->totals_dev);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_moments(lb_ctx* c, double* rho, double* u, bool want_totals) {
    switch (c->prec) {
        case LB_F64: return moments_t<double>(c, rho, u, want_totals);
        case LB_F32: return moments_t<float>(c, rho, u, want_totals);
        case LB_F16S: return moments_t<__half>(c, rho, u, want_totals);
        default: return moments_t<__nv_bfloat16>(c, rho, u, want_totals);
    }
}

cudaError_t launch_faxen(lb_ctx* c, int n, const double* F, const double* a, double* U) {
    if (n == 0) return cudaSuccess;
    const double eta = c->tau_s / 3.0;
    const double inv_aL = isinf(c->a_L) ? 0.0 : 1.0 / c->a_L;
    k_faxen<<<(n + 127) / 128, 128, 0, c->stream>>>(n, F, a, inv_aL, 1.0 / (6.0 * M_PI * eta), U);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_expand(lb_ctx* c, int n, const double* pos, const double* F, const double* param, int kind,
                          int mult) {
    (void)mult;
    if (n == 0) return cudaSuccess;
    k_expand<<<(n + 127) / 128, 128, 0, c->stream>>>(pos, F, param, n, kind, c->npts, c->geom, c->pos, c->force,
                                                      c->radius, c->mobile, c->status);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_fsum(lb_ctx* c) {
    k_fsum<<<1, 1024, 0, c->stream>>>(c->force, c->npts, c->fsum);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_set_positions(lb_ctx* c, const double* pos, bool check) {
    if (c->npts == 0) return cudaSuccess;
    k_set_positions<<<(c->npts + 127) / 128, 128, 0, c->stream>>>(pos, c->npts, c->geom, check ? nullptr : c->pos,
                                                                  c->status);
    c->launches++;
    return cudaGetLastError();
}

template <typename S>
static cudaError_t convert_t(lb_ctx* c, double* out, const double* in) {
    const long long count = (long long)NQ * c->geom.V;
    const unsigned int blocks = (unsigned int)std::min<long long>((count + 255) / 256, 152LL * 32);
    if (out)
        k_convert_out<S><<<blocks, 256, 0, c->stream>>>((const S*)c->f[c->cur], count, c->inv_scale, out);
    else
        k_convert_in<S><<<blocks, 256, 0, c->stream>>>(in, count, c->scale, (S*)c->f[c->cur], c->seed);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_convert_out(lb_ctx* c, double* df) {
    switch (c->prec) {
        case LB_F64: return convert_t<double>(c, df, nullptr);
        case LB_F32: return convert_t<float>(c, df, nullptr);
        case LB_F16S: return convert_t<__half>(c, df, nullptr);
        default: return convert_t<__nv_bfloat16>(c, df, nullptr);
    }
}

cudaError_t launch_convert_in(lb_ctx* c, const double* df) {
    switch (c->prec) {
        case LB_F64: return convert_t<double>(c, nullptr, df);
        case LB_F32: return convert_t<float>(c, nullptr, df);
        case LB_F16S: return convert_t<__half>(c, nullptr, df);
        default: return convert_t<__nv_bfloat16>(c, nullptr, df);
    }
}

// Zero the spread field where it can be non-zero -- the flagged 8-site
// groups -- and the flags: each warp takes 32 tiles (one flag word per
// lane), then clears the flagged groups of each flagged tile, one site per
// lane.  The field is zero outside the flagged groups (the spread flags
// every group it adds to), so this equals zeroing all of it, at the cost
// of reading the flags (4 B per 32 sites) instead of writing 3 values a
// site.
template <typename T>
__global__ void __launch_bounds__(256) k_clear_groups(Geom g, T* __restrict__ floc, flag_t* __restrict__ flags) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned ntiles = (unsigned)g.ntiles, ntx = (unsigned)g.ntx;
    const unsigned ngroups = (ntiles + 31u) >> 5;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned* words = (unsigned*)flags;
    for (unsigned grp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; grp < ngroups; grp += nwarps) {
        const unsigned t = (grp << 5) + lane;
        const unsigned w = t < ntiles ? words[t] : 0u;
        unsigned m = __ballot_sync(0xffffffffu, w != 0u);
        if (w) words[t] = 0u;
        while (m) {
            const unsigned b = (unsigned)(__ffs(m) - 1);
            m &= m - 1u;
            const unsigned wt = __shfl_sync(0xffffffffu, w, b);
            const unsigned tile = (grp << 5) + b;
            const unsigned row = tile / ntx;  // z * ny + y
            const unsigned x = (tile - row * ntx) * TILE_X + lane;
            if (x < (unsigned)g.nx && group_flag(wt, lane)) {
                const unsigned site = row * (unsigned)g.nx + x;
                field_st(floc, site, T(0), T(0), T(0));
            }
        }
    }
}

cudaError_t launch_clear_field(lb_ctx* c) {
    const long long warps = (c->geom.ntiles + 31) / 32;
    // a warp a flag word group: the walk is a dependent load then a few
    // stores, so every group gets its own warp
    const unsigned blocks = (unsigned)std::max<long long>(1, (warps + 7) / 8);
    if (c->prec == LB_F64)
        k_clear_groups<double><<<blocks, 256, 0, c->stream>>>(c->geom, (double*)c->floc, c->flags);
    else
        k_clear_groups<float><<<blocks, 256, 0, c->stream>>>(c->geom, (float*)c->floc, c->flags);
    c->launches++;
    return cudaGetLastError();
}


cudaError_t compute_inv_aL(const int grid[3], const double R[3], const double dir[3], double* inv_aL) {
    const int blocks = 152 * 4;
    double* part = nullptr;
    cudaError_t e = cudaMalloc(&part, sizeof(double) * (blocks + 1));
    if (e != cudaSuccess) return e;
    double d[3] = {0.0, 0.0, 1.0};
    int iso = 1;
    if (dir) {
        const double nrm = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        for (int a = 0; a < 3; ++a) d[a] = dir[a] / nrm;
        iso = 0;
    }
    k_aL<<<blocks, 256>>>(grid[0], grid[1], grid[2], R[0], R[1], R[2], d[0], d[1], d[2], iso, part);
    k_sum1<<<1, 256>>>(part, blocks, part + blocks);
    double s = 0.0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(&s, part + blocks, sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(part);
    const double V = (double)grid[0] * grid[1] * grid[2];
    *inv_aL = 6.0 * M_PI / V * s;
    return e;
}

}  // namespace lbk
