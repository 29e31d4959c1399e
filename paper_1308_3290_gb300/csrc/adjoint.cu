// Kernels of the discrete adjoint of the one-layer CGPRK3 step (the paper has
// no adjoint; these transpose the Jacobian of the step of Section 3.2).
//
// With psi = A w (A = P^l S R^l, symmetric) the transposed right-hand side is
//   G_w^T lam = J(psi, lam) + (1/Re) lap lam - A[J(w, lam) - (1/Ro) J(lam, y)],
// because J(p, .) (Arakawa's enstrophy conservation, Section 4.1) and the beta
// operator J(., y) are skew-symmetric on fields that vanish on the walls.
// adj_source computes the bracket, the host applies A with the forward
// restriction / solve / prolongation kernels, and adj_stage assembles the
// transposed TVDRK3 stage (Eq. TVDRK in stage form w^(s+1) = a w^n +
// b (w^(s) + dt G(w^(s)))).
#include <cuda_runtime.h>

#include "arakawa.cuh"
#include "bounds.cuh"
#include "qg_internal.cuh"

namespace qg {
namespace {

// out = J(w, lam) - (1/Ro) J(lam, y) at the interior nodes.
template <typename T>
__global__ void adj_source_kernel(const T* __restrict__ w, const T* __restrict__ lam,
                                  T* __restrict__ out, AdjParams<T> p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (i >= p.nx || j >= p.ny) return;
    const int ld = p.ld;
    const size_t c = (size_t)j * ld + i;
    if (!(QG_IN((long long)c - ld - 1, (long long)(p.ny + 1) * ld, 111) &&
          QG_IN((long long)c + ld + 1, (long long)(p.ny + 1) * ld, 111)))
        return;
    const T* P = w + c;
    const T* Q = lam + c;
    const T pm0 = P[-1], p10 = P[1], p0m = P[-ld], p01 = P[ld];
    const T pmm = P[-ld - 1], p1m = P[-ld + 1], pm1 = P[ld - 1], p11 = P[ld + 1];
    const T qm0 = Q[-1], q10 = Q[1], q0m = Q[-ld], q01 = Q[ld];
    const T qmm = Q[-ld - 1], q1m = Q[-ld + 1], qm1 = Q[ld - 1], q11 = Q[ld + 1];
    const T jac = arakawa_sum(pm0, p10, p0m, p01, pmm, p1m, pm1, p11, qm0, q10, q0m, q01,
                              qmm, q1m, qm1, q11) * p.c_jac;
    // (1/Ro) J(lam, y): the closed form (4 c_j + c_{j+1} + c_{j-1}) / (6 Ro)
    // with c the central x difference of lam
    const T beta = (T(4) * (q10 - qm0) + (q11 - qm1) + (q1m - qmm)) * p.c_beta;
    out[c] = jac - beta;
}

// One transposed TVDRK3 stage:
//   v = J(psi, lam) + (1/Re) lap lam - phi        (phi = A of adj_source)
//   next = [next +] b lam + b dt v,  acc += a lam,  g += b dt lam.
// next may alias acc only when a = 0 (the first stage).
template <typename T>
__global__ void adj_stage_kernel(const T* __restrict__ psi, const T* __restrict__ lam,
                                 const T* __restrict__ phi, T* next, T* acc,
                                 T* __restrict__ g, AdjParams<T> p, int accumulate) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (i >= p.nx || j >= p.ny) return;
    const int ld = p.ld;
    const size_t c = (size_t)j * ld + i;
    if (!(QG_IN((long long)c - ld - 1, (long long)(p.ny + 1) * ld, 111) &&
          QG_IN((long long)c + ld + 1, (long long)(p.ny + 1) * ld, 111)))
        return;
    const T* P = psi + c;
    const T* Q = lam + c;
    const T pm0 = P[-1], p10 = P[1], p0m = P[-ld], p01 = P[ld];
    const T pmm = P[-ld - 1], p1m = P[-ld + 1], pm1 = P[ld - 1], p11 = P[ld + 1];
    const T q00 = Q[0];
    const T qm0 = Q[-1], q10 = Q[1], q0m = Q[-ld], q01 = Q[ld];
    const T qmm = Q[-ld - 1], q1m = Q[-ld + 1], qm1 = Q[ld - 1], q11 = Q[ld + 1];
    const T jac = arakawa_sum(pm0, p10, p0m, p01, pmm, p1m, pm1, p11, qm0, q10, q0m, q01,
                              qmm, q1m, qm1, q11) * p.c_jac;
    const T lap = (q10 + qm0 - T(2) * q00) * p.c_lapx + (q01 + q0m - T(2) * q00) * p.c_lapy;
    const T v = jac + lap - phi[c];
    T out = p.b * (q00 + p.dt * v);
    if (accumulate) out += next[c];
    if (p.a != T(0)) acc[c] += p.a * q00;
    next[c] = out;
    g[c] += p.b * p.dt * q00;
}

// out = -dx dy lap psi: dE/dpsi of E = 1/2 dx dy sum over edges of the squared
// one-sided differences (= -1/2 dx dy sum psi lap psi with zero walls).
template <typename T>
__global__ void energy_source_kernel(const T* __restrict__ psi, T* __restrict__ out,
                                     AdjParams<T> p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (i >= p.nx || j >= p.ny) return;
    const int ld = p.ld;
    const size_t c = (size_t)j * ld + i;
    if (!(QG_IN((long long)c - ld - 1, (long long)(p.ny + 1) * ld, 111) &&
          QG_IN((long long)c + ld + 1, (long long)(p.ny + 1) * ld, 111)))
        return;
    const T* P = psi + c;
    const T lap = (P[1] + P[-1] - T(2) * P[0]) * p.inv_dx2 + (P[ld] + P[-ld] - T(2) * P[0]) * p.inv_dy2;
    out[c] = -p.dxdy * lap;
}

// dense[(j-1)(nx-1) + i-1] += scale * padded[j ld + i] over the interior.
template <typename T>
__global__ void add_to_dense_kernel(T* __restrict__ dense, const T* __restrict__ padded,
                                    T scale, int nx, int ny, int ld) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (i >= nx || j >= ny) return;
    if (!(QG_IN((long long)(j - 1) * (nx - 1) + (i - 1), (long long)(nx - 1) * (ny - 1), 112) &&
          QG_IN((long long)j * ld + i, (long long)(ny + 1) * ld, 112)))
        return;
    dense[(size_t)(j - 1) * (nx - 1) + (i - 1)] += scale * padded[(size_t)j * ld + i];
}

dim3 grid_for(int nx, int ny, dim3 b) {
    return dim3((nx - 1 + b.x - 1) / b.x, (ny - 1 + b.y - 1) / b.y);
}

}  // namespace

template <typename T>
cudaError_t launch_adj_source(const T* w, const T* lam, T* out, const AdjParams<T>& p,
                              cudaStream_t s) {
    const dim3 b(32, 8);
    adj_source_kernel<T><<<grid_for(p.nx, p.ny, b), b, 0, s>>>(w, lam, out, p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adj_stage(const T* psi, const T* lam, const T* phi, T* next, T* acc, T* g,
                             const AdjParams<T>& p, bool accumulate, cudaStream_t s) {
    const dim3 b(32, 8);
    adj_stage_kernel<T><<<grid_for(p.nx, p.ny, b), b, 0, s>>>(psi, lam, phi, next, acc, g, p,
                                                              accumulate ? 1 : 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_energy_source(const T* psi, T* out, const AdjParams<T>& p, cudaStream_t s) {
    const dim3 b(32, 8);
    energy_source_kernel<T><<<grid_for(p.nx, p.ny, b), b, 0, s>>>(psi, out, p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_add_to_dense(T* dense, const T* padded, double scale, int nx, int ny, int ld,
                                cudaStream_t s) {
    const dim3 b(32, 8);
    add_to_dense_kernel<T><<<grid_for(nx, ny, b), b, 0, s>>>(dense, padded, (T)scale, nx, ny, ld);
    return cudaGetLastError();
}

#define QG_INST(T)                                                                          \
    template cudaError_t launch_adj_source<T>(const T*, const T*, T*, const AdjParams<T>&,  \
                                              cudaStream_t);                                \
    template cudaError_t launch_adj_stage<T>(const T*, const T*, const T*, T*, T*, T*,      \
                                             const AdjParams<T>&, bool, cudaStream_t);      \
    template cudaError_t launch_energy_source<T>(const T*, T*, const AdjParams<T>&,         \
                                                 cudaStream_t);                             \
    template cudaError_t launch_add_to_dense<T>(T*, const T*, double, int, int, int,        \
                                                cudaStream_t);
QG_INST(float)
QG_INST(double)
#undef QG_INST

QG_BOUNDS_QUERY(bounds_site_adjoint)

}  // namespace qg
