// The nine-point Arakawa combination of Section 4.1 (Eqs. j1, j2, j3),
// shared by the unfused stage kernels and the adjoint kernels.
#pragma once

namespace qg {

// The nine-point Arakawa combination J1 + J2 + J3 (without 1/(4 dx dy) and
// the 1/3), for psi values p.. and q values q.. at offsets (di, dj), m = -1.
template <typename T>
__device__ __forceinline__ T arakawa_sum(T pm0, T p10, T p0m, T p01, T pmm,
                                         T p1m, T pm1, T p11, T qm0, T q10,
                                         T q0m, T q01, T qmm, T q1m, T qm1,
                                         T q11) {
    const T j1 = -(q10 - qm0) * (p01 - p0m) + (q01 - q0m) * (p10 - pm0);
    const T j2 = -q10 * (p11 - p1m) + qm0 * (pm1 - pmm) + q01 * (p11 - pm1) -
                 q0m * (p1m - pmm);
    const T j3 = -q11 * (p01 - p10) + qmm * (pm0 - p0m) + qm1 * (p01 - pm0) -
                 q1m * (p10 - p0m);
    return j1 + j2 + j3;
}

}  // namespace qg
