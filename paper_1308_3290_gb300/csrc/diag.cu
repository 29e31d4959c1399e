// FP64 diagnostics of a basin state: the basin-integrated kinetic energy
// (Section 5.2, E = 1/2 iint |grad psi|^2, one-sided differences on grid
// edges), the enstrophy 1/2 iint w^2, and max(|psi_x|, |psi_y|) (the
// denominator of the CFL time step, Eq. dt).
//
// Differences are formed in the working precision and squared and summed in
// FP64.  Each CTA covers a fixed strided set of nodes and reduces through a
// fixed shared-memory tree; one CTA then folds the per-CTA results in index
// order, so the result is bitwise reproducible run to run.
#include <cuda_runtime.h>

#include "bounds.cuh"
#include "qg_internal.cuh"

namespace qg {
namespace {

constexpr int kDiagThreads = 256;
constexpr int kDiagBlocks = 304;  // 2 per SM on a 152-SM GB300

template <typename T>
__global__ void __launch_bounds__(kDiagThreads)
diag_partial_kernel(const T* __restrict__ psi, const T* __restrict__ w, int nx,
                    int ny, int ld, double* __restrict__ partial) {
    __shared__ double sh[5][kDiagThreads];
    double sx = 0.0, sy = 0.0, sw = 0.0, ux = 0.0, uy = 0.0;
    const long total = (long)nx * ny;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % nx), j = (int)(idx / nx);
        const size_t c = (size_t)j * ld + i;
        const long long n = (long long)(ny + 1) * ld;
        if (!(QG_IN((long long)c + ld, n, 101) && QG_IN((long long)c + 1, n, 101) &&
              (i < 1 || j < 1 || (QG_IN((long long)c - ld, n, 102) && QG_IN((long long)c - 1, n, 102)))))
            continue;
        if (j >= 1) {
            const double d = (double)(psi[c + 1] - psi[c]);
            sx += d * d;
        }
        if (i >= 1) {
            const double d = (double)(psi[c + ld] - psi[c]);
            sy += d * d;
        }
        if (i >= 1 && j >= 1) {
            const double v = (double)w[c];
            sw += v * v;
            ux = fmax(ux, fabs((double)(psi[c + 1] - psi[c - 1])));
            uy = fmax(uy, fabs((double)(psi[c + ld] - psi[c - ld])));
        }
    }
    sh[0][threadIdx.x] = sx;
    sh[1][threadIdx.x] = sy;
    sh[2][threadIdx.x] = sw;
    sh[3][threadIdx.x] = ux;
    sh[4][threadIdx.x] = uy;
    __syncthreads();
    for (int s = kDiagThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
            sh[2][threadIdx.x] += sh[2][threadIdx.x + s];
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + s]);
            sh[4][threadIdx.x] = fmax(sh[4][threadIdx.x], sh[4][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 5) partial[blockIdx.x * 5 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kDiagThreads)
diag_final_kernel(const double* __restrict__ partial, int nblocks,
                  double* __restrict__ out) {
    __shared__ double sh[5][kDiagThreads];
    double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        a[0] += partial[b * 5 + 0];
        a[1] += partial[b * 5 + 1];
        a[2] += partial[b * 5 + 2];
        a[3] = fmax(a[3], partial[b * 5 + 3]);
        a[4] = fmax(a[4], partial[b * 5 + 4]);
    }
    for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int s = kDiagThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
            sh[2][threadIdx.x] += sh[2][threadIdx.x + s];
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + s]);
            sh[4][threadIdx.x] = fmax(sh[4][threadIdx.x], sh[4][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 5) out[threadIdx.x] = sh[threadIdx.x][0];
}

// acc += c0 out[0] + c1 out[1]: the kinetic energy of Section 5.2 from the
// two edge sums of diag_final_kernel, scaled, added in FP64 by one thread.
__global__ void energy_add_kernel(const double* __restrict__ out, double c0, double c1,
                                  double* __restrict__ acc) {
    if (threadIdx.x == 0 && blockIdx.x == 0) acc[0] += c0 * out[0] + c1 * out[1];
}

}  // namespace

int diag_blocks() { return kDiagBlocks; }

QG_BOUNDS_QUERY(bounds_site_diag)

cudaError_t launch_energy_add(const double* out, double c0, double c1, double* acc,
                              cudaStream_t s) {
    energy_add_kernel<<<1, 32, 0, s>>>(out, c0, c1, acc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_diagnostics(const T* psi, const T* w, int nx, int ny, int ld,
                               double dx, double dy, double* partial,
                               int nblocks, double* out, cudaStream_t s) {
    (void)dx;
    (void)dy;
    diag_partial_kernel<T><<<nblocks, kDiagThreads, 0, s>>>(psi, w, nx, ny, ld, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final_kernel<<<1, kDiagThreads, 0, s>>>(partial, nblocks, out);
    return cudaGetLastError();
}

template cudaError_t launch_diagnostics<float>(const float*, const float*, int, int,
                                               int, double, double, double*, int,
                                               double*, cudaStream_t);
template cudaError_t launch_diagnostics<double>(const double*, const double*, int,
                                                int, int, double, double, double*,
                                                int, double*, cudaStream_t);

}  // namespace qg
