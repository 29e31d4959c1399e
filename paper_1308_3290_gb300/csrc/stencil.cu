// Fine-grid stage and mapping operators.
//
// fine_stage: one TVDRK3 stage (Section 4.2, Eq. TVDRK) of the one-layer
// vorticity equation on the fine grid, with the Arakawa Jacobian
// (Section 4.1, Eqs. ja1, j1-j3), the beta term J(psi, y)/Ro, the 5-point
// dissipation (1/Re) lap w and the wind forcing (Section 2.1, Eq. ge divided
// by Ro).  restrict / prolong: the mapping operators of Section 3.1 (Eqs. res
// and pro), l levels at once.
#include <cuda_runtime.h>

#include "arakawa.cuh"
#include "bounds.cuh"
#include "qg_internal.cuh"

namespace qg {
namespace {

template <typename T>
__global__ void fine_stage_kernel(const T* __restrict__ psi,
                                  const T* __restrict__ w, const T* wn,
                                  T* wout, const T* __restrict__ frow,
                                  const T* __restrict__ f2d, StageParams<T> p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (i >= p.nx || j >= p.ny) return;
    const int ld = p.ld;
    const size_t c = (size_t)j * ld + i;
    const T* P = psi + c;
    const T* Q = w + c;
    const T pm0 = P[-1], p10 = P[1], p0m = P[-ld], p01 = P[ld];
    const T pmm = P[-ld - 1], p1m = P[-ld + 1], pm1 = P[ld - 1], p11 = P[ld + 1];
    const T q00 = Q[0];
    const T qm0 = Q[-1], q10 = Q[1], q0m = Q[-ld], q01 = Q[ld];
    const T qmm = Q[-ld - 1], q1m = Q[-ld + 1], qm1 = Q[ld - 1], q11 = Q[ld + 1];
    const T jac = arakawa_sum(pm0, p10, p0m, p01, pmm, p1m, pm1, p11, qm0, q10,
                              q0m, q01, qmm, q1m, qm1, q11) * p.c_jac;
    // (1/Ro) J(psi, y) = (4 c_j + c_{j+1} + c_{j-1}) / (6 Ro),
    // c = (psi_{i+1} - psi_{i-1}) / (2 dx): Arakawa's form with q = y.
    const T beta = (T(4) * (p10 - pm0) + (p11 - pm1) + (p1m - pmm)) * p.c_beta;
    const T lap = (q10 + qm0 - T(2) * q00) * p.c_lapx + (q01 + q0m - T(2) * q00) * p.c_lapy;
    const T F = f2d ? f2d[c] : frow[j];
    const T G = -jac - beta + lap + F;
    T v = p.b * (q00 + p.dt * G);
    if (p.a != T(0)) v += p.a * wn[c];
    wout[c] = v;
}

// Two-layer stage (Section 2.2, Eq. ge-non with Q_i = q_i - y):
//   G_1 = -J(psi_1, Q_1) - J(psi_1, y) + A lap w_1 + amp sin(2 pi y)
//   G_2 = -J(psi_2, Q_2) - J(psi_2, y) + A lap w_2 - sigma w_2
// with w_i recovered from Eq. pv-non at every node of the 5-point stencil.
template <typename T>
__global__ void fine_stage2_kernel(const T* __restrict__ psi1,
                                   const T* __restrict__ psi2,
                                   const T* __restrict__ q1,
                                   const T* __restrict__ q2, const T* qn1,
                                   const T* qn2, T* out1, T* out2,
                                   const T* __restrict__ frow,
                                   StageParams2<T> p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (i >= p.nx || j >= p.ny) return;
    const int ld = p.ld;
    const size_t c = (size_t)j * ld + i;
    auto w1 = [&](size_t o) { return (q1[o] - p.f1 * (psi2[o] - psi1[o])) * p.inv_Ro; };
    auto w2 = [&](size_t o) { return (q2[o] - p.f2 * (psi1[o] - psi2[o])) * p.inv_Ro; };
#pragma unroll
    for (int layer = 0; layer < 2; ++layer) {
        const T* P = (layer == 0 ? psi1 : psi2) + c;
        const T* Q = (layer == 0 ? q1 : q2) + c;
        const T pm0 = P[-1], p10 = P[1], p0m = P[-ld], p01 = P[ld];
        const T pmm = P[-ld - 1], p1m = P[-ld + 1], pm1 = P[ld - 1], p11 = P[ld + 1];
        const T q00 = Q[0];
        const T qm0 = Q[-1], q10 = Q[1], q0m = Q[-ld], q01 = Q[ld];
        const T qmm = Q[-ld - 1], q1m = Q[-ld + 1], qm1 = Q[ld - 1], q11 = Q[ld + 1];
        const T jac = arakawa_sum(pm0, p10, p0m, p01, pmm, p1m, pm1, p11, qm0, q10,
                                  q0m, q01, qmm, q1m, qm1, q11) * p.c_jac;
        const T beta = (T(4) * (p10 - pm0) + (p11 - pm1) + (p1m - pmm)) * p.c_beta;
        T wc, wl, wr, wd, wu;
        if (layer == 0) {
            wc = w1(c); wl = w1(c - 1); wr = w1(c + 1); wd = w1(c - ld); wu = w1(c + ld);
        } else {
            wc = w2(c); wl = w2(c - 1); wr = w2(c + 1); wd = w2(c - ld); wu = w2(c + ld);
        }
        // walls: w = 0 (free slip); the formula gives 0 there since Q = psi = 0
        const T lap = (wr + wl - T(2) * wc) * p.A_dx2 + (wu + wd - T(2) * wc) * p.A_dy2;
        const T src = (layer == 0) ? frow[j] : -p.sigma * wc;
        const T G = -jac - beta + lap + src;
        T v = p.b * (q00 + p.dt * G);
        if (p.a != T(0)) v += p.a * (layer == 0 ? qn1 : qn2)[c];
        (layer == 0 ? out1 : out2)[c] = v;
    }
}

// R^l as one hat-weighted sum: with f = 2^l, the composed full weighting has
// separable weights (f - |d|)/f^2 per direction for |d| < f.
template <typename T>
__global__ void restrict_kernel(const T* __restrict__ fine, int ldf,
                                T* __restrict__ coarse, int ldc, int mx,
                                int my, int levels) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int J = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (I >= mx || J >= my) return;
    const int f = 1 << levels;
    const T* base = fine + (size_t)(f * J) * ldf + f * I;
    // the fine grid has (f my + 1) rows of pitch ldf
    const long long fn = (long long)(f * my + 1) * ldf;
    T acc = T(0);
    for (int dj = -(f - 1); dj <= f - 1; ++dj) {
        const T* row = base + (ptrdiff_t)dj * ldf;
        T racc = T(0);
        for (int di = -(f - 1); di <= f - 1; ++di) {
            const long long o = (long long)(f * J + dj) * ldf + f * I + di;
            if (QG_IN(o, fn, 41)) racc += T(f - (di < 0 ? -di : di)) * row[di];
        }
        acc += T(f - (dj < 0 ? -dj : dj)) * racc;
    }
    const T inv = T(1) / (T(f) * T(f) * T(f) * T(f));
    if (QG_IN((long long)J * ldc + I, (long long)(my + 1) * ldc, 42))
        coarse[(size_t)J * ldc + I] = acc * inv;
}

// P^l as bilinear interpolation from the coarse nodes around each fine node.
template <typename T>
__global__ void prolong_kernel(const T* __restrict__ coarse, int ldc,
                               T* __restrict__ fine, int ldf, int nx, int ny,
                               int levels) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (i >= nx || j >= ny) return;
    const int f = 1 << levels;
    const int I = i >> levels, J = j >> levels;
    const T a = T(i & (f - 1)) / T(f);
    const T b = T(j & (f - 1)) / T(f);
    const T* C = coarse + (size_t)J * ldc + I;
    // the coarse grid has (ny >> levels) + 1 rows of pitch ldc
    if (!QG_IN((long long)(J + 1) * ldc + I + 1, (long long)((ny >> levels) + 1) * ldc, 43))
        return;
    const T v = (T(1) - a) * (T(1) - b) * C[0] + a * (T(1) - b) * C[1] +
                (T(1) - a) * b * C[ldc] + a * b * C[ldc + 1];
    if (QG_IN((long long)j * ldf + i, (long long)(ny + 1) * ldf, 44))
        fine[(size_t)j * ldf + i] = v;
}

}  // namespace

template <typename T>
cudaError_t launch_fine_stage(const T* psi, const T* w, const T* wn, T* wout,
                              const T* frow, const T* f2d,
                              const StageParams<T>& p, cudaStream_t s) {
    const dim3 block(32, 8);
    const dim3 grid((p.nx - 1 + 31) / 32, (p.ny - 1 + 7) / 8);
    fine_stage_kernel<T><<<grid, block, 0, s>>>(psi, w, wn, wout, frow, f2d, p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fine_stage2(const T* psi1, const T* psi2, const T* q1,
                               const T* q2, const T* qn1, const T* qn2,
                               T* out1, T* out2, const T* frow,
                               const StageParams2<T>& p, cudaStream_t s) {
    const dim3 block(32, 8);
    const dim3 grid((p.nx - 1 + 31) / 32, (p.ny - 1 + 7) / 8);
    fine_stage2_kernel<T><<<grid, block, 0, s>>>(psi1, psi2, q1, q2, qn1, qn2,
                                                  out1, out2, frow, p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const T* fine, int ldf, T* coarse, int ldc, int mx,
                            int my, int levels, cudaStream_t s) {
    const dim3 block(32, 8);
    const dim3 grid((mx - 1 + 31) / 32, (my - 1 + 7) / 8);
    restrict_kernel<T><<<grid, block, 0, s>>>(fine, ldf, coarse, ldc, mx, my, levels);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong(const T* coarse, int ldc, T* fine, int ldf, int nx,
                           int ny, int levels, cudaStream_t s) {
    const dim3 block(32, 8);
    const dim3 grid((nx - 1 + 31) / 32, (ny - 1 + 7) / 8);
    prolong_kernel<T><<<grid, block, 0, s>>>(coarse, ldc, fine, ldf, nx, ny, levels);
    return cudaGetLastError();
}

// psi at fine node (i, j) prolonged `levels` times from the elliptic grid c:
// bilinear interpolation at spacing 2^-levels (Eq. pro applied l times).
template <typename T>
__device__ __forceinline__ T prolonged_at(const T* __restrict__ c, int ldc, int i, int j,
                                          int levels) {
    if (levels == 0) return c[(size_t)j * ldc + i];
    const int f = 1 << levels;
    const int I = i >> levels, J = j >> levels;
    const int di = i & (f - 1), dj = j & (f - 1);
    const T a = T(di) / T(f), b = T(dj) / T(f);
    const T* r0 = c + (size_t)J * ldc + I;
    const T v00 = r0[0];
    const T v10 = di ? r0[1] : T(0);
    const T v01 = dj ? r0[ldc] : T(0);
    const T v11 = (di && dj) ? r0[ldc + 1] : T(0);
    return (T(1) - b) * ((T(1) - a) * v00 + a * v10) + b * ((T(1) - a) * v01 + a * v11);
}

// Eq. dt's denominator: max over interior fine nodes of |psi_x| and |psi_y|
// (central differences) of psi prolonged `LV` times.  One thread per coarse
// cell: it interpolates the fine rows y = JF-1 .. JF+F of columns
// x = IF-1 .. IF+F from the 4 x 4 coarse patch around the cell (zero outside
// the grid; those values only reach wall nodes, which are skipped), keeps
// three rows, and takes the differences of the cell's F x F nodes.  The block
// maximum is max-ed into *umax as the bits of a non-negative double (bit
// order = value order), so the result does not depend on the block order.
template <typename T, int LV>
__global__ void cfl_max_kernel(const T* __restrict__ psi, int ldp, int nx, int ny,
                               double inv2dx, double inv2dy, unsigned long long* umax) {
    constexpr int F = 1 << LV, W = F + 2;
    __shared__ double red[32];
    // maxima of |psi(x+1) - psi(x-1)| and |psi(y+1) - psi(y-1)| in the
    // working precision (FP64 arithmetic per node is slow on this GPU); the
    // scaling by 1/(2 dx), 1/(2 dy) is monotone, so it is applied once
    T ax = T(0), ay = T(0);
    const int mx = nx >> LV, my = ny >> LV;
    const long ncell = (long)mx * my;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < ncell;
         e += (long)gridDim.x * blockDim.x) {
        const int I = (int)(e % mx), J = (int)(e / mx);
        if constexpr (LV == 0) {   // the fine psi itself: one node per thread
            if (I < 1 || J < 1) continue;
            const T* p = psi + (size_t)J * ldp + I;
            ax = fmax(ax, fabs(p[1] - p[-1]));
            ay = fmax(ay, fabs(p[ldp] - p[-ldp]));
            continue;
        }
        T c[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int Jr = J - 1 + r, Iq = I - 1 + q;
                c[r][q] = (Jr >= 0 && Jr <= my && Iq >= 0 && Iq <= mx)
                              ? psi[(size_t)Jr * ldp + Iq] : T(0);
            }
        T row[3][W];
#pragma unroll
        for (int yy = 0; yy < F + 2; ++yy) {
            const int y = J * F - 1 + yy;
            // patch row of the lower coarse line and the weight (J F is a
            // multiple of F, so both depend on yy only)
            const int jr = 1 + ((yy - 1) >> LV);
            const T b = T((yy - 1) & (F - 1)) / T(F);
            T* rv = row[yy % 3];
#pragma unroll
            for (int xx = 0; xx < W; ++xx) {
                const int iq = 1 + ((xx - 1) >> LV);
                const T a = T((xx - 1) & (F - 1)) / T(F);
                const T lo = (T(1) - a) * c[jr][iq] + (a > T(0) ? a * c[jr][iq + 1] : T(0));
                const T hi = (b > T(0)) ? (T(1) - a) * c[jr + 1][iq] +
                                              (a > T(0) ? a * c[jr + 1][iq + 1] : T(0))
                                        : T(0);
                rv[xx] = (T(1) - b) * lo + b * hi;
            }
            if (yy >= 2) {
                const int yc = y - 1;                    // the row whose differences are ready
                if (yc >= 1 && yc <= ny - 1) {
                    const T* up = row[yy % 3];
                    const T* mid = row[(yy + 2) % 3];
                    const T* dn = row[(yy + 1) % 3];
#pragma unroll
                    for (int xx = 1; xx <= F; ++xx) {
                        const int x = I * F - 1 + xx;
                        if (x < 1 || x > nx - 1) continue;
                        ax = fmax(ax, fabs(mid[xx + 1] - mid[xx - 1]));
                        ay = fmax(ay, fabs(up[xx] - dn[xx]));
                    }
                }
            }
        }
    }
    double m = fmax((double)ax * inv2dx, (double)ay * inv2dy);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) atomicMax(umax, (unsigned long long)__double_as_longlong(m));
    }
}

template <typename T>
cudaError_t launch_cfl_max(const T* psi, int ldp, int nx, int ny, int levels, double dx,
                           double dy, unsigned long long* umax, cudaStream_t s) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long ncell = (long)(nx >> levels) * (ny >> levels);
    long blocks = (ncell + 255) / 256;
    if (blocks > 8L * nsm) blocks = 8L * nsm;
    const double ix = 0.5 / dx, iy = 0.5 / dy;
    switch (levels) {
        case 0: cfl_max_kernel<T, 0><<<(int)blocks, 256, 0, s>>>(psi, ldp, nx, ny, ix, iy, umax); break;
        case 1: cfl_max_kernel<T, 1><<<(int)blocks, 256, 0, s>>>(psi, ldp, nx, ny, ix, iy, umax); break;
        case 2: cfl_max_kernel<T, 2><<<(int)blocks, 256, 0, s>>>(psi, ldp, nx, ny, ix, iy, umax); break;
        case 3: cfl_max_kernel<T, 3><<<(int)blocks, 256, 0, s>>>(psi, ldp, nx, ny, ix, iy, umax); break;
        default: cfl_max_kernel<T, 4><<<(int)blocks, 256, 0, s>>>(psi, ldp, nx, ny, ix, iy, umax); break;
    }
    return cudaGetLastError();
}

template <typename T>
__global__ void accumulate_kernel(double* __restrict__ acc, const T* __restrict__ src, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x)
        acc[e] += (double)src[e];
}

template <typename T>
__global__ void mean_out_kernel(T* __restrict__ dense, const double* __restrict__ acc, int ldacc,
                                double scale, int nx, int ny, int levels) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (i >= nx || j >= ny) return;
    dense[(size_t)(j - 1) * (nx - 1) + (i - 1)] = (T)(scale * prolonged_at(acc, ldacc, i, j, levels));
}

// dense = scale * acc (fine nodes) + y_j: the time-mean potential vorticity
template <typename T>
__global__ void mean_q_out_kernel(T* __restrict__ dense, const double* __restrict__ acc, int ld,
                                  double scale, int nx, int ny, double y0, double dy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (i >= nx || j >= ny) return;
    dense[(size_t)(j - 1) * (nx - 1) + (i - 1)] =
        (T)(scale * acc[(size_t)j * ld + i] + (y0 + dy * (double)j));
}

template <typename T>
cudaError_t launch_mean_q_out(T* dense, const double* acc, int ld, double scale, int nx, int ny,
                              double y0, double dy, cudaStream_t s) {
    const dim3 block(32, 8);
    const dim3 grid((nx - 1 + 31) / 32, (ny - 1 + 7) / 8);
    mean_q_out_kernel<T><<<grid, block, 0, s>>>(dense, acc, ld, scale, nx, ny, y0, dy);
    return cudaGetLastError();
}
template cudaError_t launch_mean_q_out<float>(float*, const double*, int, double, int, int, double,
                                              double, cudaStream_t);
template cudaError_t launch_mean_q_out<double>(double*, const double*, int, double, int, int,
                                               double, double, cudaStream_t);

template <typename T>
cudaError_t launch_accumulate(double* acc, const T* src, size_t n, cudaStream_t s) {
    size_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    accumulate_kernel<T><<<(int)blocks, 256, 0, s>>>(acc, src, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mean_out(T* dense, const double* acc, int ldacc, double scale, int nx,
                            int ny, int levels, cudaStream_t s) {
    const dim3 block(32, 8);
    const dim3 grid((nx - 1 + 31) / 32, (ny - 1 + 7) / 8);
    mean_out_kernel<T><<<grid, block, 0, s>>>(dense, acc, ldacc, scale, nx, ny, levels);
    return cudaGetLastError();
}

// dense (nym1 rows of nxm1) <-> padded interior.  The dense side (often
// pinned host memory reached over the C2C link) moves in 16-byte vectors
// of the flat array when it is 16-byte aligned, the padded side element by
// element; both are row-contiguous, so both sides coalesce.
template <typename W>
__global__ void repack_kernel(W* __restrict__ dst, const W* __restrict__ src, int nxm1, int nym1,
                              int ld, int to_padded) {
    constexpr int V = 16 / sizeof(W);
    const long n = (long)nxm1 * nym1;
    const W* dense_r = to_padded ? src : nullptr;
    W* dense_w = to_padded ? nullptr : dst;
    const bool vec = ((reinterpret_cast<uintptr_t>(to_padded ? (const void*)src : (const void*)dst)
                       & 15) == 0);
    const long nv = vec ? n / V : 0;
    auto pad = [&](long e) { const int j = (int)(e / nxm1); return (size_t)(j + 1) * ld + (e - (long)j * nxm1) + 1; };
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < nv;
         g += (long)gridDim.x * blockDim.x) {
        W v[V];
        if (to_padded) {
            const uint4 u = reinterpret_cast<const uint4*>(dense_r)[g];
            memcpy(v, &u, 16);
#pragma unroll
            for (int k = 0; k < V; ++k) dst[pad(g * V + k)] = v[k];
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) v[k] = src[pad(g * V + k)];
            uint4 u;
            memcpy(&u, v, 16);
            reinterpret_cast<uint4*>(dense_w)[g] = u;
        }
    }
    for (long e = nv * V + (long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
        if (to_padded) dst[pad(e)] = src[e];
        else dst[e] = src[pad(e)];
    }
}

// A pointer the GPU can dereference for `ptr` (device memory, or pinned host
// memory reached over the C2C link), or null for pageable host memory.
static const void* device_view(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return ptr;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer;
    return nullptr;
}

static cudaError_t repack(void* dst, const void* src, int nxm1, int nym1, int ld, size_t esz,
                          bool to_padded, cudaStream_t s) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long n = (long)nxm1 * nym1;
    long blocks = (n + 255) / 256;
    if (blocks > 16L * nsm) blocks = 16L * nsm;
    if (esz == 8)
        repack_kernel<double><<<(int)blocks, 256, 0, s>>>(static_cast<double*>(dst),
                                                          static_cast<const double*>(src), nxm1,
                                                          nym1, ld, to_padded ? 1 : 0);
    else
        repack_kernel<float><<<(int)blocks, 256, 0, s>>>(static_cast<float*>(dst),
                                                         static_cast<const float*>(src), nxm1,
                                                         nym1, ld, to_padded ? 1 : 0);
    return cudaGetLastError();
}

// Device buffers and pinned host buffers (read or written in place over the
// C2C link, which beats a DMA copy plus a device repack) are repacked by a
// kernel; pageable host buffers go through 2-D copies.
cudaError_t copy_in(void* padded, int ld, const void* dense, int nxm1, int nym1,
                    size_t esz, cudaStream_t s) {
    if (const void* v = device_view(dense)) return repack(padded, v, nxm1, nym1, ld, esz, true, s);
    char* dst = static_cast<char*>(padded) + (size_t)(ld + 1) * esz;
    return cudaMemcpy2DAsync(dst, (size_t)ld * esz, dense, (size_t)nxm1 * esz,
                             (size_t)nxm1 * esz, nym1, cudaMemcpyDefault, s);
}

cudaError_t copy_out(void* dense, const void* padded, int ld, int nxm1, int nym1,
                     size_t esz, cudaStream_t s) {
    if (const void* v = device_view(dense))
        return repack(const_cast<void*>(v), padded, nxm1, nym1, ld, esz, false, s);
    const char* src = static_cast<const char*>(padded) + (size_t)(ld + 1) * esz;
    return cudaMemcpy2DAsync(dense, (size_t)nxm1 * esz, src, (size_t)ld * esz,
                             (size_t)nxm1 * esz, nym1, cudaMemcpyDefault, s);
}

#define QG_INST(T)                                                                  \
    template cudaError_t launch_fine_stage<T>(const T*, const T*, const T*, T*,     \
                                              const T*, const T*,                   \
                                              const StageParams<T>&, cudaStream_t); \
    template cudaError_t launch_fine_stage2<T>(const T*, const T*, const T*,        \
                                               const T*, const T*, const T*, T*,    \
                                               T*, const T*,                        \
                                               const StageParams2<T>&,              \
                                               cudaStream_t);                       \
    template cudaError_t launch_restrict<T>(const T*, int, T*, int, int, int, int,  \
                                            cudaStream_t);                          \
    template cudaError_t launch_prolong<T>(const T*, int, T*, int, int, int, int,   \
                                           cudaStream_t);                            \
    template cudaError_t launch_cfl_max<T>(const T*, int, int, int, int, double,     \
                                           double, unsigned long long*, cudaStream_t); \
    template cudaError_t launch_accumulate<T>(double*, const T*, size_t, cudaStream_t); \
    template cudaError_t launch_mean_out<T>(T*, const double*, int, double, int, int,  \
                                            int, cudaStream_t);
QG_INST(float)
QG_INST(double)
#undef QG_INST

QG_BOUNDS_QUERY(bounds_site_stencil)

}  // namespace qg
