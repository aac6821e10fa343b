// lb_kernels.cu -- sm_103a kernels of the forced D3Q19 MRT lattice
// Boltzmann method with singular point forces, and their launchers.
//
//   k_collide   fused pull-stream + moment-space collision with the
//               second-order forcing term (Sec. II, Eq. fiexp); one thread
//               per site, one warp per 32-site x-row tile; reads the
//               localised force only in tiles flagged by k_spread, then
//               clears them.
//   k_spread    regularised point forces onto the lattice (Sec. III,
//               Eq. deltadef): one thread per (point, stencil node),
//               atomic accumulation.
//   k_gather    velocity interpolated with the same kernel (Sec. IV);
//               one warp per point, two stencil nodes per lane, each node
//               rebuilt from its pulled populations; optionally the Faxen
//               update with the a_L subtraction (Eq. a_Ldefn).
//   k_moments   rho, u fields and FP64 totals (Eq. macrovariables2).
#include <math.h>

#include <algorithm>

#include "../../include/lb.h"
#include "lb_internal.h"

namespace lbk {

constexpr int CS_WARPS = 4;  // tiles (warps) per block of the site kernels
constexpr int CS_THREADS = CS_WARPS * 32;

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

template <typename S>
static Pops<S> pops(void* base, long long V) {
    Pops<S> p;
    for (int i = 0; i < NQ; ++i) p.p[i] = (S*)base + (size_t)i * (size_t)V;
    return p;
}

// Site kernels: block = 4 warps, one warp per 32-site x-row tile; grid =
// (tiles per row, ceil(ny / 4), nz).  No division in the index math.
static dim3 site_grid(const Geom& g) {
    return dim3((unsigned)g.ntx, (unsigned)((g.ny + CS_WARPS - 1) / CS_WARPS), (unsigned)g.nz);
}

// ------------------------------------------------------------ k_collide
// NY consecutive y rows per thread (all loads of the NY sites issued
// first).  The half format is handled in its scaled units throughout.
// Occupancy bound (blocks of 128 threads per SM), swept on GB300 at 256^3:
// the 4- and 2-byte formats are fastest at 12 (42 registers; 8-10 were
// 2-10 % slower, 14 spills); FP64 at 8.
// FIELD = false: a lattice without point forces (no flag or field access).
template <typename S, bool WALLS, int NY, bool FIELD>
__global__ void __launch_bounds__(CS_THREADS, (NY == 1 ? (sizeof(S) == 8 ? 8 : 12) : 4))
k_collide(const Pops<S> src, const Pops<S> dst, const typename Store<S>::T* __restrict__ floc,
          const unsigned* __restrict__ flags, Geom g, Coef<typename Store<S>::T> k,
          UForce<typename Store<S>::T> fu, float scale, float inv_scale, unsigned seed) {
    using T = typename Store<S>::T;
    constexpr bool SC = Store<S>::kScaled;
    const int y0 = (blockIdx.y * CS_WARPS + threadIdx.y) * NY;
    if (y0 >= g.ny) return;  // uniform per warp
    const int z = blockIdx.z, lane = threadIdx.x;
    const int x = blockIdx.x * TILE_X + lane;
    const unsigned V = (unsigned)g.V;
    unsigned fl[NY];
#pragma unroll
    for (int r = 0; r < NY; ++r) {
        const unsigned tile = ((unsigned)z * (unsigned)g.ny + (unsigned)(y0 + r)) * (unsigned)g.ntx + blockIdx.x;
        fl[r] = (FIELD && y0 + r < g.ny) ? __ldg(flags + tile) : 0u;
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
#pragma unroll
            for (int r = 0; r < NY; ++r) {
                if (y0 + r >= g.ny) break;
                const unsigned site = n[r].c + n[r].x;
                T Fx = fu.F[0], Fy = fu.F[1], Fz = fu.F[2];
                if (FIELD && fl[r]) {  // after the population loads, so both are in flight together
                    const T s = SC ? (T)scale : T(1);
                    Fx += floc[site] * s;
                    Fy += floc[V + site] * s;
                    Fz += floc[2 * V + site] * s;
                }
                T o[NQ];
                collide19<T, Store<S>::kCompensate, SC>(f[r], Fx, Fy, Fz, k, o, (T)inv_scale);
                unsigned rn = rng_seed(site, seed);
#pragma unroll
                for (int i = 0; i < NQ; ++i) Store<S>::st(dst.p[i], site, o[i], rng_next(rn));
            }
        }
    }
}

// Clear the consumed force tiles (k_clear_tiles runs after k_collide): the
// collide kernel only reads the field, so it never stores to a line whose
// load may still be in flight.
template <typename T>
__global__ void __launch_bounds__(256)
k_clear_tiles(Geom g, T* __restrict__ floc, unsigned* __restrict__ flags, const unsigned* __restrict__ list,
              unsigned* __restrict__ ctr) {
    clear_listed_tiles<T>(g, floc, flags, list, ctr, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctr[1], 1u) == gridDim.x - 1) {  // last block: reset the list
            ctr[0] = 0u;
            ctr[1] = 0u;
        }
    }
}

// ------------------------------------------------------------- k_spread
template <typename T, bool WALLS>
__global__ void __launch_bounds__(256)
k_spread(const double* __restrict__ pos, const double* __restrict__ force, int npts, T* __restrict__ floc,
         unsigned* __restrict__ flags, unsigned* __restrict__ list, unsigned* __restrict__ ctr, Geom g) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)npts * 64) return;
    const int s = (int)(t >> 6), node = (int)(t & 63);
    const int i = node & 3, j = (node >> 2) & 3, k = node >> 4;
    const double X = pos[3 * s], Y = pos[3 * s + 1], Z = pos[3 * s + 2];
    const int nxg = stencil_base(X) + i, nyg = stencil_base(Y) + j, nzg = stencil_base(Z) + k;
    const int z = wrap_node(nzg, g.nz);
    if (WALLS && is_solid(g, z)) return;
    const int x = wrap_node(nxg, g.nx), y = wrap_node(nyg, g.ny);
    const T wx = peskin_phi((T)((double)nxg - X));
    const T wy = peskin_phi((T)((double)nyg - Y));
    const T wz = peskin_phi((T)((double)nzg - Z));
    const T w = wx * wy * wz;
    const long long site = ((long long)z * g.ny + y) * g.nx + x;
    atomicAdd(floc + site, (T)force[3 * s] * w);
    atomicAdd(floc + g.V + site, (T)force[3 * s + 1] * w);
    atomicAdd(floc + 2 * g.V + site, (T)force[3 * s + 2] * w);
    mark_tile(flags, list, ctr, (unsigned)(((long long)z * g.ny + y) * g.ntx + x / TILE_X));
}

// Position wrapped into [0, n).
__device__ __forceinline__ double wrap_pos(double r, int n) {
    const double L = (double)n;
    r = r - L * floor(r / L);
    if (r >= L || r < 0.0) r = 0.0;
    return r;
}

// ------------------------------------------------------------- k_gather
// v at the n points (query mode) or at every colloid with the position
// update (update mode).  One warp per point.
template <typename S, bool WALLS>
__global__ void __launch_bounds__(128)
k_gather(const Pops<S> src, const typename Store<S>::T* __restrict__ floc, Geom g, UForce<typename Store<S>::T> fu,
         float inv_scale, int n, const double* __restrict__ qpos, double* __restrict__ vout,
         double* __restrict__ upos, const double* __restrict__ force, const double* __restrict__ radius,
         const int* __restrict__ mobile, double inv_6pi_eta, double inv_aL) {
    using T = typename Store<S>::T;
    const int s = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (s >= n) return;
    const bool update = (upos != nullptr);
    if (update && !mobile[s]) return;
    const int lane = threadIdx.x & 31;
    const double* P = update ? upos + 3 * s : qpos + 3 * s;
    const double X = wrap_pos(P[0], g.nx), Y = wrap_pos(P[1], g.ny), Z = wrap_pos(P[2], g.nz);
    const int bx = stencil_base(X), by = stencil_base(Y), bz = stencil_base(Z);
    const unsigned V = (unsigned)g.V;
    T acc[3] = {T(0), T(0), T(0)};
    for (int h = 0; h < 2; ++h) {
        const int node = lane + 32 * h;
        const int i = node & 3, j = (node >> 2) & 3, k = node >> 4;
        const int x = wrap_node(bx + i, g.nx), y = wrap_node(by + j, g.ny), z = wrap_node(bz + k, g.nz);
        if (WALLS && is_solid(g, z)) continue;  // v = 0 on solid nodes
        const T w = peskin_phi((T)((double)(bx + i) - X)) * peskin_phi((T)((double)(by + j) - Y)) *
                    peskin_phi((T)((double)(bz + k) - Z));
        const Nbr nb = neighbours(g, x, y, z);
        const unsigned site = nb.c + nb.x;
        T f[NQ];
        pull19<S, WALLS>(src, nb, f);
        unscale19<S>(f, inv_scale);
        const T Fx = fu.F[0] + floc[site], Fy = fu.F[1] + floc[V + site], Fz = fu.F[2] + floc[2 * V + site];
        T drho, vx, vy, vz;
        macro19<T, Store<S>::kCompensate>(f, Fx, Fy, Fz, drho, vx, vy, vz);
        acc[0] += w * vx;
        acc[1] += w * vy;
        acc[2] += w * vz;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        for (int a = 0; a < 3; ++a) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], off);
    if (lane != 0) return;
    if (!update) {
        for (int a = 0; a < 3; ++a) vout[3 * s + a] = (double)acc[a];
        return;
    }
    const double c = (1.0 / radius[s] - inv_aL) * inv_6pi_eta;
    const int nn[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a)
        upos[3 * s + a] = wrap_pos(P[a] + (double)acc[a] + force[3 * s + a] * c, nn[a]);
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
            const T Fx = fu.F[0] + floc[site], Fy = fu.F[1] + floc[V + site], Fz = fu.F[2] + floc[2 * V + site];
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

// Colloid update with the learned correction: R += v(R) + F (1/a - 1/a_L) /
// (6 pi eta) + y |F| / (6 pi eta a), y the network output in units of the
// Stokes velocity of the colloid.
__global__ void k_corrected_update(int n, const double* __restrict__ v, const float* __restrict__ y,
                                   const double* __restrict__ F, const double* __restrict__ a,
                                   const int* __restrict__ mobile, double inv_aL, double inv_6pi_eta, Geom g,
                                   double* __restrict__ pos) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n || !mobile[t]) return;
    const double f0 = F[3 * t], f1 = F[3 * t + 1], f2 = F[3 * t + 2];
    const double c = (1.0 / a[t] - inv_aL) * inv_6pi_eta;
    const double v0 = sqrt(f0 * f0 + f1 * f1 + f2 * f2) * inv_6pi_eta / a[t];
    const int nn[3] = {g.nx, g.ny, g.nz};
    for (int k = 0; k < 3; ++k)
        pos[3 * t + k] = wrap_pos(pos[3 * t + k] + v[3 * t + k] + F[3 * t + k] * c + (double)y[3 * t + k] * v0, nn[k]);
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

__global__ void k_set_positions(const double* __restrict__ in, int npts, Geom g, double* __restrict__ pos,
                                int* __restrict__ status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npts) return;
    const int nn[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a) {
        const double r = in[3 * t + a];
        if (!isfinite(r)) {
            atomicOr(status, 1);
            return;
        }
        pos[3 * t + a] = wrap_pos(r, nn[a]);
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

// ------------------------------------------------------------ launchers
static bool has_walls(const lb_ctx* c) { return c->geom.wall_lo >= 0 || c->geom.wall_hi >= 0; }
static dim3 site_block() { return dim3(TILE_X, CS_WARPS, 1); }

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
    const T* floc = (const T*)c->floc;
    const bool field = c->npts > 0;
#define LB_COLLIDE(W, FD)                                                                                       \
    k_collide<S, W, NY, FD><<<grid, site_block(), 0, c->stream>>>(src, dst, floc, c->flags, c->geom, k, fu, c->scale, \
                                                                c->inv_scale, c->seed)
    if (has_walls(c)) {
        if (field) LB_COLLIDE(true, true);
        else LB_COLLIDE(true, false);
    } else {
        if (field) LB_COLLIDE(false, true);
        else LB_COLLIDE(false, false);
    }
#undef LB_COLLIDE
    c->seed = c->seed * 747796405u + 2891336453u;  // next step's rounding seed
    c->launches++;
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

template <typename T>
static cudaError_t spread_t(lb_ctx* c) {
    const long long threads = (long long)c->npts * 64;
    const unsigned int blocks = (unsigned int)((threads + 255) / 256);
    if (has_walls(c))
        k_spread<T, true><<<blocks, 256, 0, c->stream>>>(c->pos, c->force, c->npts, (T*)c->floc, c->flags,
                                                          c->tile_list, c->tile_ctr, c->geom);
    else
        k_spread<T, false><<<blocks, 256, 0, c->stream>>>(c->pos, c->force, c->npts, (T*)c->floc, c->flags,
                                                           c->tile_list, c->tile_ctr, c->geom);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_spread(lb_ctx* c) {
    if (c->npts == 0) return cudaSuccess;
    return c->prec == LB_F64 ? spread_t<double>(c) : spread_t<float>(c);
}

template <typename S>
static cudaError_t gather_t(lb_ctx* c, int n, const double* qpos, double* vout, bool update) {
    using T = typename Store<S>::T;
    const UForce<T> fu = uniform_force<T>(c);
    const double eta = c->tau_s / 3.0;
    const double inv_6pi_eta = 1.0 / (6.0 * M_PI * eta);
    const double inv_aL = isinf(c->a_L) ? 0.0 : 1.0 / c->a_L;
    const unsigned int blocks = (unsigned int)((n + 3) / 4);
    const Pops<S> src = pops<S>(c->f[c->cur], c->geom.V);
    double* upos = update ? c->pos : nullptr;
    if (has_walls(c))
        k_gather<S, true><<<blocks, 128, 0, c->stream>>>(src, (const T*)c->floc, c->geom, fu, c->inv_scale, n, qpos,
                                                          vout, upos, c->force, c->radius, c->mobile, inv_6pi_eta,
                                                          inv_aL);
    else
        k_gather<S, false><<<blocks, 128, 0, c->stream>>>(src, (const T*)c->floc, c->geom, fu, c->inv_scale, n, qpos,
                                                           vout, upos, c->force, c->radius, c->mobile, inv_6pi_eta,
                                                           inv_aL);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_gather(lb_ctx* c, int n, const double* qpos, double* vout, bool update) {
    if (n == 0) return cudaSuccess;
    switch (c->prec) {
        case LB_F64: return gather_t<double>(c, n, qpos, vout, update);
        case LB_F32: return gather_t<float>(c, n, qpos, vout, update);
        case LB_F16S: return gather_t<__half>(c, n, qpos, vout, update);
        default: return gather_t<__nv_bfloat16>(c, n, qpos, vout, update);
    }
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

cudaError_t launch_corrected_update(lb_ctx* c) {
    const double eta = c->tau_s / 3.0;
    const double inv_aL = isinf(c->a_L) ? 0.0 : 1.0 / c->a_L;
    k_corrected_update<<<(c->npts + 127) / 128, 128, 0, c->stream>>>(c->npts, c->corr_v, c->corr_y, c->force,
                                                                    c->radius, c->mobile, inv_aL,
                                                                    1.0 / (6.0 * M_PI * eta), c->geom, c->pos);
    c->launches++;
    return cudaGetLastError();
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

cudaError_t launch_set_positions(lb_ctx* c, const double* pos) {
    if (c->npts == 0) return cudaSuccess;
    k_set_positions<<<(c->npts + 127) / 128, 128, 0, c->stream>>>(pos, c->npts, c->geom, c->pos, c->status);
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

cudaError_t launch_clear_field(lb_ctx* c) {
    cudaError_t e = cudaMemsetAsync(c->floc, 0, 3 * (size_t)c->geom.V * arith_bytes(c->prec), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->flags, 0, sizeof(unsigned) * (size_t)c->geom.ntiles, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->tile_ctr, 0, sizeof(unsigned) * 2, c->stream);
    return e;
}

cudaError_t launch_clear_tiles(lb_ctx* c) {
    // a point flags at most 32 tiles (4 x 4 node rows, two x-tiles each):
    // size the grid for that many 32-site tiles, at most 2 blocks per SM
    const long long lanes = std::min<long long>((long long)c->npts * 32 * 32, c->geom.ntiles * 32);
    const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>(152 * 2, (lanes + 255) / 256));
    if (c->prec == LB_F64)
        k_clear_tiles<double><<<blocks, 256, 0, c->stream>>>(c->geom, (double*)c->floc, c->flags, c->tile_list,
                                                             c->tile_ctr);
    else
        k_clear_tiles<float><<<blocks, 256, 0, c->stream>>>(c->geom, (float*)c->floc, c->flags, c->tile_list,
                                                            c->tile_ctr);
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
