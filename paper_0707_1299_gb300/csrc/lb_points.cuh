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
