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
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbk {

constexpr int NQ = 19;
constexpr int TILE_X = 32;  // one warp of x-consecutive sites = one force tile

// Lattice geometry, passed by value to every kernel.
struct Geom {
    int nx, ny, nz;
    int ntx;            // tiles per x-row: ceil(nx / 32)
    long long V;        // nx * ny * nz
    long long ntiles;   // ntx * ny * nz
    int wall_lo, wall_hi;  // solid z-planes, -1 = none
};

__device__ __forceinline__ bool is_solid(const Geom& g, int z) {
    return z == g.wall_lo || z == g.wall_hi;
}

// ----------------------------------------------------------- storage types
// df is stored as S and handled in arithmetic type T.  The half-precision
// formats store df * scale (a power of two) to keep df out of subnormals.
template <typename S> struct Store;
template <> struct Store<double> {
    using T = double;
    static __device__ __forceinline__ double ld(const double* p, long long i, float) { return __ldg(p + i); }
    static __device__ __forceinline__ void st(double* p, long long i, double v, float) { __stcs(p + i, v); }
};
template <> struct Store<float> {
    using T = float;
    static __device__ __forceinline__ float ld(const float* p, long long i, float) { return __ldg(p + i); }
    static __device__ __forceinline__ void st(float* p, long long i, float v, float) { __stcs(p + i, v); }
};
template <> struct Store<__half> {
    using T = float;
    static __device__ __forceinline__ float ld(const __half* p, long long i, float inv_scale) {
        return __half2float(__ldg(p + i)) * inv_scale;
    }
    static __device__ __forceinline__ void st(__half* p, long long i, float v, float scale) {
        p[i] = __float2half_rn(v * scale);
    }
};
template <> struct Store<__nv_bfloat16> {
    using T = float;
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p, long long i, float inv_scale) {
        return __bfloat162float(__ldg(p + i)) * inv_scale;
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, long long i, float v, float scale) {
        p[i] = __float2bfloat16_rn(v * scale);
    }
};

// ------------------------------------------------------------ pull stream
// Neighbour coordinates of (x, y, z) with periodic wrap.
struct Nbr {
    long long c, ym, yp, zm, zp, zmym, zmyp, zpym, zpyp;  // row offsets ((z*ny+y)*nx)
    int x, xm, xp;
    bool solid_zm, solid_zp;
};

__device__ __forceinline__ Nbr neighbours(const Geom& g, int x, int y, int z) {
    Nbr n;
    const int ym = (y == 0) ? g.ny - 1 : y - 1, yp = (y == g.ny - 1) ? 0 : y + 1;
    const int zm = (z == 0) ? g.nz - 1 : z - 1, zp = (z == g.nz - 1) ? 0 : z + 1;
    n.x = x;
    n.xm = (x == 0) ? g.nx - 1 : x - 1;
    n.xp = (x == g.nx - 1) ? 0 : x + 1;
    const long long nx = g.nx, ny = g.ny;
    n.c = ((long long)z * ny + y) * nx;
    n.ym = ((long long)z * ny + ym) * nx;
    n.yp = ((long long)z * ny + yp) * nx;
    n.zm = ((long long)zm * ny + y) * nx;
    n.zp = ((long long)zp * ny + y) * nx;
    n.zmym = ((long long)zm * ny + ym) * nx;
    n.zmyp = ((long long)zm * ny + yp) * nx;
    n.zpym = ((long long)zp * ny + ym) * nx;
    n.zpyp = ((long long)zp * ny + yp) * nx;
    n.solid_zm = is_solid(g, zm);
    n.solid_zp = is_solid(g, zp);
    return n;
}

// df_i(x) = df*_i(x - c_i); where x - c_i is a solid node the population
// bounces back: df_i(x) = df*_ibar(x).
template <typename S, bool WALLS>
__device__ __forceinline__ void pull19(const S* __restrict__ src, long long V, const Nbr& n, float inv_scale,
                                       typename Store<S>::T f[NQ]) {
    using St = Store<S>;
    const long long own = n.c + n.x;
    f[0] = St::ld(src, 0 * V + own, inv_scale);
    f[1] = St::ld(src, 1 * V + n.c + n.xm, inv_scale);
    f[2] = St::ld(src, 2 * V + n.c + n.xp, inv_scale);
    f[3] = St::ld(src, 3 * V + n.ym + n.x, inv_scale);
    f[4] = St::ld(src, 4 * V + n.yp + n.x, inv_scale);
    f[7] = St::ld(src, 7 * V + n.ym + n.xm, inv_scale);
    f[8] = St::ld(src, 8 * V + n.yp + n.xp, inv_scale);
    f[9] = St::ld(src, 9 * V + n.yp + n.xm, inv_scale);
    f[10] = St::ld(src, 10 * V + n.ym + n.xp, inv_scale);
    if (!WALLS || !n.solid_zm) {
        f[5] = St::ld(src, 5 * V + n.zm + n.x, inv_scale);
        f[11] = St::ld(src, 11 * V + n.zm + n.xm, inv_scale);
        f[14] = St::ld(src, 14 * V + n.zm + n.xp, inv_scale);
        f[15] = St::ld(src, 15 * V + n.zmym + n.x, inv_scale);
        f[18] = St::ld(src, 18 * V + n.zmyp + n.x, inv_scale);
    } else {
        f[5] = St::ld(src, 6 * V + own, inv_scale);
        f[11] = St::ld(src, 12 * V + own, inv_scale);
        f[14] = St::ld(src, 13 * V + own, inv_scale);
        f[15] = St::ld(src, 16 * V + own, inv_scale);
        f[18] = St::ld(src, 17 * V + own, inv_scale);
    }
    if (!WALLS || !n.solid_zp) {
        f[6] = St::ld(src, 6 * V + n.zp + n.x, inv_scale);
        f[12] = St::ld(src, 12 * V + n.zp + n.xp, inv_scale);
        f[13] = St::ld(src, 13 * V + n.zp + n.xm, inv_scale);
        f[16] = St::ld(src, 16 * V + n.zpyp + n.x, inv_scale);
        f[17] = St::ld(src, 17 * V + n.zpym + n.x, inv_scale);
    } else {
        f[6] = St::ld(src, 5 * V + own, inv_scale);
        f[12] = St::ld(src, 11 * V + own, inv_scale);
        f[13] = St::ld(src, 14 * V + own, inv_scale);
        f[16] = St::ld(src, 15 * V + own, inv_scale);
        f[17] = St::ld(src, 18 * V + own, inv_scale);
    }
}

// ------------------------------------------------------------- moments
template <typename T>
struct Moments {
    T drho, jx, jy, jz;        // sum df, sum df c
    T pxx, pyy, pzz, pxy, pxz, pyz;  // sum df c_a c_b
};

template <typename T>
__device__ __forceinline__ Moments<T> moments19(const T f[NQ]) {
    Moments<T> m;
    const T a12 = f[1] + f[2], a34 = f[3] + f[4], a56 = f[5] + f[6];
    const T d78 = f[7] + f[8], d910 = f[9] + f[10], d1112 = f[11] + f[12], d1314 = f[13] + f[14];
    const T d1516 = f[15] + f[16], d1718 = f[17] + f[18];
    m.drho = f[0] + a12 + a34 + a56 + d78 + d910 + d1112 + d1314 + d1516 + d1718;
    const T e78 = f[7] - f[8], e910 = f[9] - f[10], e1112 = f[11] - f[12], e1314 = f[13] - f[14];
    const T e1516 = f[15] - f[16], e1718 = f[17] - f[18];
    m.jx = (f[1] - f[2]) + e78 + e910 + e1112 + e1314;
    m.jy = (f[3] - f[4]) + e78 - e910 + e1516 + e1718;
    m.jz = (f[5] - f[6]) + e1112 - e1314 + e1516 - e1718;
    m.pxx = a12 + d78 + d910 + d1112 + d1314;
    m.pyy = a34 + d78 + d910 + d1516 + d1718;
    m.pzz = a56 + d1112 + d1314 + d1516 + d1718;
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

// Post-collision df* from the pulled df and the local force density F:
//   A = j + F,  v = (j + F/2) / rho,  S = sum df Q,
//   X = S - rho vv,  Y = vF + Fv,
//   B = S - om_s dev(X - tau_s Y) - (om_b / 3) tr(X - tau_b Y) 1,
//   df*_i = w_i [drho + 3 A.c_i + 4.5 c_i.B.c_i - 1.5 tr B].
template <typename T>
__device__ __forceinline__ void collide19(const T f[NQ], T Fx, T Fy, T Fz, const Coef<T>& k, T out[NQ]) {
    const Moments<T> m = moments19(f);
    const T third = T(1) / T(3);
    const T rho = T(1) + m.drho;
    const T irho = T(1) / rho;
    const T vx = (m.jx + T(0.5) * Fx) * irho;
    const T vy = (m.jy + T(0.5) * Fy) * irho;
    const T vz = (m.jz + T(0.5) * Fz) * irho;
    // S = P - (drho/3) 1 ; X = S - rho vv ; Y = vF + Fv
    const T sxx = m.pxx - third * m.drho, syy = m.pyy - third * m.drho, szz = m.pzz - third * m.drho;
    const T xxx = sxx - rho * vx * vx, xyy = syy - rho * vy * vy, xzz = szz - rho * vz * vz;
    const T xxy = m.pxy - rho * vx * vy, xxz = m.pxz - rho * vx * vz, xyz = m.pyz - rho * vy * vz;
    const T yxx = T(2) * vx * Fx, yyy = T(2) * vy * Fy, yzz = T(2) * vz * Fz;
    const T yxy = vx * Fy + Fx * vy, yxz = vx * Fz + Fx * vz, yyz = vy * Fz + Fy * vz;
    const T trX = xxx + xyy + xzz, trY = yxx + yyy + yzz;
    const T dev_tr = third * (trX - k.tau_s * trY);
    const T iso = third * k.om_b * (trX - k.tau_b * trY);
    const T bxx = sxx - k.om_s * (xxx - k.tau_s * yxx - dev_tr) - iso;
    const T byy = syy - k.om_s * (xyy - k.tau_s * yyy - dev_tr) - iso;
    const T bzz = szz - k.om_s * (xzz - k.tau_s * yzz - dev_tr) - iso;
    const T bxy = m.pxy - k.om_s * (xxy - k.tau_s * yxy);
    const T bxz = m.pxz - k.om_s * (xxz - k.tau_s * yxz);
    const T byz = m.pyz - k.om_s * (xyz - k.tau_s * yyz);
    const T ax = m.jx + Fx, ay = m.jy + Fy, az = m.jz + Fz;

    const T base = m.drho - T(1.5) * (bxx + byy + bzz);
    const T w0 = T(1) / T(3), w1 = T(1) / T(18), w2 = T(1) / T(36);
    out[0] = w0 * base;
    const T hx = base + T(4.5) * bxx, hy = base + T(4.5) * byy, hz = base + T(4.5) * bzz;
    const T ax3 = T(3) * ax, ay3 = T(3) * ay, az3 = T(3) * az;
    out[1] = w1 * (hx + ax3);
    out[2] = w1 * (hx - ax3);
    out[3] = w1 * (hy + ay3);
    out[4] = w1 * (hy - ay3);
    out[5] = w1 * (hz + az3);
    out[6] = w1 * (hz - az3);
    // (s1, s2) face diagonals in plane (a, b): base + 4.5 (Baa + Bbb) + 9 s1 s2 Bab + 3 (s1 Aa + s2 Ab)
    const T pxy_ = base + T(4.5) * (bxx + byy), pxz_ = base + T(4.5) * (bxx + bzz), pyz_ = base + T(4.5) * (byy + bzz);
    const T qxy = T(9) * bxy, qxz = T(9) * bxz, qyz = T(9) * byz;
    out[7] = w2 * (pxy_ + qxy + (ax3 + ay3));
    out[8] = w2 * (pxy_ + qxy - (ax3 + ay3));
    out[9] = w2 * (pxy_ - qxy + (ax3 - ay3));
    out[10] = w2 * (pxy_ - qxy - (ax3 - ay3));
    out[11] = w2 * (pxz_ + qxz + (ax3 + az3));
    out[12] = w2 * (pxz_ + qxz - (ax3 + az3));
    out[13] = w2 * (pxz_ - qxz + (ax3 - az3));
    out[14] = w2 * (pxz_ - qxz - (ax3 - az3));
    out[15] = w2 * (pyz_ + qyz + (ay3 + az3));
    out[16] = w2 * (pyz_ + qyz - (ay3 + az3));
    out[17] = w2 * (pyz_ - qyz + (ay3 - az3));
    out[18] = w2 * (pyz_ - qyz - (ay3 - az3));
}

// drho = rho - 1 and v = (j + F/2) / rho, Eq. (macrovariables2).
template <typename T>
__device__ __forceinline__ void macro19(const T f[NQ], T Fx, T Fy, T Fz, T& drho, T& vx, T& vy, T& vz) {
    const Moments<T> m = moments19(f);
    drho = m.drho;
    const T rho = T(1) + m.drho;
    const T irho = T(1) / rho;
    vx = (m.jx + T(0.5) * Fx) * irho;
    vy = (m.jy + T(0.5) * Fy) * irho;
    vz = (m.jz + T(0.5) * Fz) * irho;
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
    // k in [-1, n + 2); also correct for n < 4 where it may wrap twice
    int r = k % n;
    return r < 0 ? r + n : r;
}

}  // namespace lbk
