// gp2s_kernel_math.cuh -- device evaluation of the kernel pieces shared by the assembly, value and
// adjoint kernels: the Wendland taper (Eq. 3 and the "C2" reading) and its derivative.
#pragma once

#include <cuda_runtime.h>

namespace gp2s {

// phi(t) for t = |xi - xj| / r; zero for t >= 1 (strict support, Eq. 3).
//   kind 1 (Eq. 3):        (1-t)^8 (32 t^3 + 25 t^2 + 8 t + 1)
//   kind 0, d <= 3 (C2 reading):  (1-t)^4 (4 t + 1)
//   kind 0, d == 4 (C2 reading):  (1-t)^5 (5 t + 1)
template <class T>
__device__ __forceinline__ T wendland(int kind, int d, T t)
{
    if (!(t < T(1))) return T(0);
    if (t < T(0)) t = T(0);
    const T u = T(1) - t;
    const T u2 = u * u;
    if (kind == 1) {
        const T u4 = u2 * u2;
        return (u4 * u4) * (((T(32) * t + T(25)) * t + T(8)) * t + T(1));
    }
    if (d <= 3) return (u2 * u2) * (T(4) * t + T(1));
    return (u2 * u2 * u) * (T(5) * t + T(1));
}

// d phi / d t.
template <class T>
__device__ __forceinline__ T wendland_dt(int kind, int d, T t)
{
    if (!(t < T(1))) return T(0);
    if (t < T(0)) t = T(0);
    const T u = T(1) - t;
    const T u2 = u * u;
    if (kind == 1) {
        const T u7 = u2 * u2 * u2 * u;
        return T(-22) * t * u7 * ((T(16) * t + T(7)) * t + T(1));
    }
    if (d <= 3) return T(-20) * t * (u2 * u);
    return T(-30) * t * (u2 * u2);
}

// phi'(t) / t, finite at t = 0 (each form's derivative carries a factor t).
template <class T>
__device__ __forceinline__ T wendland_dt_over_t(int kind, int d, T t)
{
    if (!(t < T(1))) return T(0);
    if (t < T(0)) t = T(0);
    const T u = T(1) - t;
    const T u2 = u * u;
    if (kind == 1) {
        const T u7 = u2 * u2 * u2 * u;
        return T(-22) * u7 * ((T(16) * t + T(7)) * t + T(1));
    }
    if (d <= 3) return T(-20) * (u2 * u);
    return T(-30) * (u2 * u2);
}

}  // namespace gp2s
