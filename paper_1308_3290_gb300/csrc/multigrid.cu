// Geometric multigrid for the elliptic sub-problem (Section 3: the CGP step
// does not depend on which Poisson solver runs on the coarse grid; the paper
// names the V-cycle multigrid as the solver of choice where sine transforms
// do not apply).
//
// lap_h psi = f on an mx x my grid of intervals with psi = 0 on the walls
// (the 5-point operator whose eigenvalues Eq. ialpha gives, Section 4.3,
// with the grid's own spacings).  One V(2,2)
// cycle:
//   - two red-black Gauss-Seidel sweeps (each point solves its own 5-point
//     equation for the current neighbours);
//   - the residual r = f - lap_h psi restricted to the next grid by full
//     weighting, the operator of Eq. res (fine wall residuals are zero);
//   - the coarse-grid correction (recursively, from a zero guess);
//   - the correction prolonged by bilinear interpolation, the operator of
//     Eq. pro, and added;
//   - two more sweeps.
// Grids are halved until the shorter side has 2 intervals; there the
// unknowns form one line and the 5-point equations a tridiagonal system,
// solved exactly (Thomas algorithm).  The finest levels are one
// launch per operation; the levels from `tail` down run in one CTA out of
// shared memory.
#include <cuda_runtime.h>

#include <mutex>

#include "bounds.cuh"
#include "qg_internal.cuh"

namespace qg {
namespace {

constexpr int kPre = 2, kPost = 2;

template <typename T>
struct Grid {
    T* psi;
    const T* rhs;
    int mx, my, ld, ldr;   // intervals, pitch of psi, pitch of rhs
    T cx, cy;              // 1/dx^2, 1/dy^2
};

// ---- one operation on one grid, for a range of threads ---------------
// (used by the per-level kernels with the whole launch, and by the tail
// kernel with the CTA)

template <typename T>
__device__ __forceinline__ void rb_half(const Grid<T>& g, int color, int tid, int nthr) {
    const int hw = g.mx / 2;                   // points of one colour per row (upper bound)
    const int n = hw * (g.my - 1);
    const T inv = T(1) / (T(2) * (g.cx + g.cy));
    for (int e = tid; e < n; e += nthr) {
        const int j = 1 + e / hw;
        const int i = 2 * (e % hw) + (((1 + j) & 1) == color ? 1 : 2);
        if (i > g.mx - 1) continue;
        const long long o = (long long)j * g.ld + i, n = (long long)(g.my + 1) * g.ld;
        if (!(QG_IN(o - g.ld, n, 91) && QG_IN(o + g.ld, n, 91) &&
              QG_IN((long long)j * g.ldr + i, (long long)(g.my + 1) * g.ldr, 92)))
            continue;
        T* p = g.psi + (size_t)j * g.ld + i;
        const T f = g.rhs[(size_t)j * g.ldr + i];
        p[0] = (g.cx * (p[-1] + p[1]) + g.cy * (p[-g.ld] + p[g.ld]) - f) * inv;
    }
}

template <typename T>
__device__ __forceinline__ T residual_at(const Grid<T>& g, int i, int j) {
    if (i < 1 || j < 1 || i > g.mx - 1 || j > g.my - 1) return T(0);
    const long long o = (long long)j * g.ld + i, n = (long long)(g.my + 1) * g.ld;
    if (!(QG_IN(o - g.ld, n, 93) && QG_IN(o + g.ld, n, 93) &&
          QG_IN((long long)j * g.ldr + i, (long long)(g.my + 1) * g.ldr, 93)))
        return T(0);
    const T* p = g.psi + (size_t)j * g.ld + i;
    const T lap = g.cx * (p[-1] + p[1] - T(2) * p[0]) + g.cy * (p[-g.ld] + p[g.ld] - T(2) * p[0]);
    return g.rhs[(size_t)j * g.ldr + i] - lap;
}

// coarse f = R(f - lap_h psi) (Eq. res on the residual), coarse psi = 0
template <typename T>
__device__ __forceinline__ void restrict_residual(const Grid<T>& g, T* cf, T* cpsi, int cmx,
                                                  int cmy, int cld, int tid, int nthr) {
    const int n = (cmx - 1) * (cmy - 1);
    for (int e = tid; e < n; e += nthr) {
        const int I = 1 + e % (cmx - 1), J = 1 + e / (cmx - 1);
        const int i = 2 * I, j = 2 * J;
        if (!QG_IN((long long)J * cld + I, (long long)(cmy + 1) * cld, 94)) continue;
        const T c = residual_at(g, i, j);
        const T ed = residual_at(g, i - 1, j) + residual_at(g, i + 1, j) +
                     residual_at(g, i, j - 1) + residual_at(g, i, j + 1);
        const T co = residual_at(g, i - 1, j - 1) + residual_at(g, i + 1, j - 1) +
                     residual_at(g, i - 1, j + 1) + residual_at(g, i + 1, j + 1);
        cf[(size_t)J * cld + I] = (T(4) * c + T(2) * ed + co) * T(0.0625);
        cpsi[(size_t)J * cld + I] = T(0);
    }
}

// fine psi += P(coarse psi) (Eq. pro; coarse wall values are zero)
template <typename T>
__device__ __forceinline__ void prolong_add(const Grid<T>& g, const T* cpsi, int cld, int tid,
                                            int nthr) {
    const int n = (g.mx - 1) * (g.my - 1);
    for (int e = tid; e < n; e += nthr) {
        const int i = 1 + e % (g.mx - 1), j = 1 + e / (g.mx - 1);
        const int I = i >> 1, J = j >> 1;
        const long long cn = (long long)((g.my >> 1) + 1) * cld;
        if (!(QG_IN((long long)J * cld + I, cn, 95) && QG_IN((long long)(J + 1) * cld + I + 1, cn, 95) &&
              QG_IN((long long)j * g.ld + i, (long long)(g.my + 1) * g.ld, 96)))
            continue;
        const T* c = cpsi + (size_t)J * cld + I;
        T v;
        if (!(i & 1) && !(j & 1)) v = c[0];
        else if (!(j & 1)) v = T(0.5) * (c[0] + c[1]);
        else if (!(i & 1)) v = T(0.5) * (c[0] + c[cld]);
        else v = T(0.25) * (c[0] + c[1] + c[cld] + c[cld + 1]);
        g.psi[(size_t)j * g.ld + i] += v;
    }
}

// The coarsest grid: a shorter side of 2 intervals leaves one line of n <= 7
// unknowns u_k (the sides are within a factor 4); the walls beside it are
// zero, so its 5-point equations read  c u_{k-1} + d u_k + c u_{k+1} = f_k,
// d = -2 (cx + cy), c the coefficient along the line.  Forward elimination
// and back substitution (one thread; |d| > 2c keeps it stable).
template <typename T>
__device__ void line_solve(const Grid<T>& g) {
    const bool along_y = g.mx == 2;
    const int n = along_y ? g.my - 1 : g.mx - 1;
    if (n > 8) return;
    const T c = along_y ? g.cy : g.cx;
    const T d = -T(2) * (g.cx + g.cy);
    auto u = [&](int k) -> T& {
        return along_y ? g.psi[(size_t)(k + 1) * g.ld + 1] : g.psi[(size_t)g.ld + k + 1];
    };
    auto f = [&](int k) -> T {
        return along_y ? g.rhs[(size_t)(k + 1) * g.ldr + 1] : g.rhs[(size_t)g.ldr + k + 1];
    };
    T cs[8];
    T cprev = T(0), uprev = T(0);
    for (int k = 0; k < n; ++k) {
        const T den = d - c * cprev;
        cs[k] = c / den;
        uprev = (f(k) - c * uprev) / den;
        u(k) = uprev;
        cprev = cs[k];
    }
    for (int k = n - 2; k >= 0; --k) u(k) -= cs[k] * u(k + 1);
}

// ---- per-level kernels ---------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(256) mg_rb_kernel(Grid<T> g, int color) {
    rb_half(g, color, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

template <typename T>
__global__ void __launch_bounds__(256) mg_restrict_kernel(Grid<T> g, T* cf, T* cpsi, int cmx,
                                                          int cmy, int cld) {
    restrict_residual(g, cf, cpsi, cmx, cmy, cld, blockIdx.x * blockDim.x + threadIdx.x,
                      gridDim.x * blockDim.x);
}

template <typename T>
__global__ void __launch_bounds__(256) mg_prolong_kernel(Grid<T> g, const T* cpsi, int cld) {
    prolong_add(g, cpsi, cld, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// rhs0 = P0 + P1 + ... (the restriction's partial planes, in that order),
// psi0 = 0 when `zero`
template <typename T>
__global__ void __launch_bounds__(256) mg_sum_kernel(MGSumParams<T> q) {
    const int n = (q.mx - 1) * (q.my - 1);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int i = 1 + e % (q.mx - 1), j = 1 + e / (q.mx - 1);
        const size_t o = (size_t)j * q.ld_in + i;
        T v = q.in[0][o];
        for (int k = 1; k < q.nin; ++k) v = v + q.in[k][o];
        q.rhs[(size_t)j * q.ld + i] = v;
        if (q.zero) q.psi[(size_t)j * q.ld + i] = T(0);
    }
}

// ---- the tail: levels t..C in one CTA, out of shared memory -------------
// On entry psi_t (global) holds the initial guess and rhs_t (global) the
// right-hand side; one V-cycle over levels t..C; psi_t is written back.
template <typename T>
__global__ void __launch_bounds__(512) mg_tail_kernel(MGTail<T> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    T* base = reinterpret_cast<T*>(smem);
    const int tid = threadIdx.x, nthr = blockDim.x;
    // smem layout: for each level k: psi[(my+1)(mx+1)], rhs[(my+1)(mx+1)]
    Grid<T> g[kMaxTail];
    size_t off = 0;
    for (int k = 0; k < a.n; ++k) {
        const int ld = a.mx[k] + 1;
        const size_t sz = (size_t)(a.my[k] + 1) * ld;
        g[k].psi = base + off;
        g[k].rhs = base + off + sz;
        g[k].mx = a.mx[k];
        g[k].my = a.my[k];
        g[k].ld = g[k].ldr = ld;
        g[k].cx = a.cx[k];
        g[k].cy = a.cy[k];
        off += 2 * sz;
    }
#ifdef QG_BOUNDS_CHECK
    {
        // the levels' arrays inside the launch's dynamic shared memory (the
        // same test in every thread)
        unsigned dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        if (!QG_IN((long long)(off * sizeof(T)) - 1, (long long)dyn, 97)) return;
    }
#endif
    for (size_t e = tid; e < off; e += nthr) base[e] = T(0);
    __syncthreads();
    {
        const int n = (a.mx[0] + 1) * (a.my[0] + 1);
        T* rhs0 = const_cast<T*>(g[0].rhs);
        for (int e = tid; e < n; e += nthr) {
            const int i = e % (a.mx[0] + 1), j = e / (a.mx[0] + 1);
            const bool in = i >= 1 && j >= 1 && i <= a.mx[0] - 1 && j <= a.my[0] - 1 &&
                            QG_IN((long long)j * a.ld + i, (long long)(a.my[0] + 1) * a.ld, 98) &&
                            QG_IN((long long)j * a.ldr + i, (long long)(a.my[0] + 1) * a.ldr, 98);
            g[0].psi[e] = in ? a.psi[(size_t)j * a.ld + i] : T(0);
            rhs0[e] = in ? a.rhs[(size_t)j * a.ldr + i] : T(0);
        }
    }
    __syncthreads();
    for (int k = 0; k + 1 < a.n; ++k) {
        for (int s = 0; s < kPre; ++s)
            for (int c = 0; c < 2; ++c) {
                rb_half(g[k], c, tid, nthr);
                __syncthreads();
            }
        restrict_residual(g[k], const_cast<T*>(g[k + 1].rhs), g[k + 1].psi, g[k + 1].mx,
                          g[k + 1].my, g[k + 1].ld, tid, nthr);
        __syncthreads();
    }
    if (tid == 0) line_solve(g[a.n - 1]);
    __syncthreads();
    for (int k = a.n - 2; k >= 0; --k) {
        prolong_add(g[k], g[k + 1].psi, g[k + 1].ld, tid, nthr);
        __syncthreads();
        for (int s = 0; s < kPost; ++s)
            for (int c = 0; c < 2; ++c) {
                rb_half(g[k], c, tid, nthr);
                __syncthreads();
            }
    }
    const int n = (a.mx[0] - 1) * (a.my[0] - 1);
    for (int e = tid; e < n; e += nthr) {
        const int i = 1 + e % (a.mx[0] - 1), j = 1 + e / (a.mx[0] - 1);
        if (!QG_IN((long long)j * a.ld + i, (long long)(a.my[0] + 1) * a.ld, 99)) continue;
        a.psi[(size_t)j * a.ld + i] = g[0].psi[(size_t)j * g[0].ld + i];
    }
}

int blocks_for(long n) {
    long b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > 4096) b = 4096;
    return (int)b;
}

}  // namespace

// The tail kernel's shared-memory limit, raised once per process to the
// most any hierarchy uses (called when a hierarchy is built, outside any
// stream capture).
cudaError_t mg_reserve_tail_smem(size_t bytes, size_t esz) {
    static std::mutex mu;             // handles on other host threads share it
    static size_t have[2] = {0, 0};
    std::lock_guard<std::mutex> lock(mu);
    const int k = esz == 8 ? 1 : 0;
    if (bytes <= have[k]) return cudaSuccess;
    const cudaError_t e =
        esz == 8 ? cudaFuncSetAttribute(mg_tail_kernel<double>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)
                 : cudaFuncSetAttribute(mg_tail_kernel<float>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have[k] = bytes;
    return e;
}

int mg_cycle_launches(int tail) { return tail * (2 * kPre + 2 * kPost + 2) + 1; }

size_t mg_tail_smem(const int* mx, const int* my, int n, size_t esz) {
    size_t s = 0;
    for (int k = 0; k < n; ++k) s += 2 * (size_t)(mx[k] + 1) * (my[k] + 1) * esz;
    return s;
}

template <typename T>
cudaError_t launch_mg_sum(const MGSumParams<T>& q, cudaStream_t s) {
    mg_sum_kernel<T><<<blocks_for((long)(q.mx - 1) * (q.my - 1)), 256, 0, s>>>(q);
    return cudaGetLastError();
}

// One V-cycle.  lv[0..nl): the grids (psi, rhs, sizes, pitches, 1/dx^2,
// 1/dy^2); the levels from `tail` on are the tail's.
template <typename T>
cudaError_t launch_mg_cycle(const MGLevelDesc<T>* lv, int nl, int tail, cudaStream_t s) {
    auto grid = [&](int k) {
        Grid<T> g;
        g.psi = lv[k].psi;
        g.rhs = lv[k].rhs;
        g.mx = lv[k].mx;
        g.my = lv[k].my;
        g.ld = lv[k].ld;
        g.ldr = lv[k].ldr;
        g.cx = lv[k].cx;
        g.cy = lv[k].cy;
        return g;
    };
    for (int k = 0; k < tail; ++k) {
        const Grid<T> g = grid(k);
        const int nb = blocks_for((long)(g.mx / 2) * (g.my - 1));
        for (int p = 0; p < kPre; ++p)
            for (int c = 0; c < 2; ++c) mg_rb_kernel<T><<<nb, 256, 0, s>>>(g, c);
        mg_restrict_kernel<T><<<blocks_for((long)(lv[k + 1].mx - 1) * (lv[k + 1].my - 1)), 256, 0,
                                s>>>(g, lv[k + 1].rhs_w, lv[k + 1].psi, lv[k + 1].mx,
                                     lv[k + 1].my, lv[k + 1].ld);
    }
    {
        MGTail<T> a = {};
        a.n = nl - tail;
        if (a.n > kMaxTail) return cudaErrorInvalidValue;
        for (int k = 0; k < a.n; ++k) {
            a.mx[k] = lv[tail + k].mx;
            a.my[k] = lv[tail + k].my;
            a.cx[k] = lv[tail + k].cx;
            a.cy[k] = lv[tail + k].cy;
        }
        a.psi = lv[tail].psi;
        a.rhs = lv[tail].rhs;
        a.ld = lv[tail].ld;
        a.ldr = lv[tail].ldr;
        const size_t sm = mg_tail_smem(a.mx, a.my, a.n, sizeof(T));
        mg_tail_kernel<T><<<1, 512, sm, s>>>(a);
    }
    for (int k = tail - 1; k >= 0; --k) {
        const Grid<T> g = grid(k);
        mg_prolong_kernel<T><<<blocks_for((long)(g.mx - 1) * (g.my - 1)), 256, 0, s>>>(
            g, lv[k + 1].psi, lv[k + 1].ld);
        const int nb = blocks_for((long)(g.mx / 2) * (g.my - 1));
        for (int p = 0; p < kPost; ++p)
            for (int c = 0; c < 2; ++c) mg_rb_kernel<T><<<nb, 256, 0, s>>>(g, c);
    }
    return cudaGetLastError();
}

QG_BOUNDS_QUERY(bounds_site_mg)

template cudaError_t launch_mg_sum<float>(const MGSumParams<float>&, cudaStream_t);
template cudaError_t launch_mg_sum<double>(const MGSumParams<double>&, cudaStream_t);
template cudaError_t launch_mg_cycle<float>(const MGLevelDesc<float>*, int, int, cudaStream_t);
template cudaError_t launch_mg_cycle<double>(const MGLevelDesc<double>*, int, int, cudaStream_t);

}  // namespace qg
