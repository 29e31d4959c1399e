// Shared-memory DST-I engine and the elliptic solver passes (Section 4.3).
//
// The paper's sine sums (Eqs. ifft-1/2, ffft-1/2) are unnormalised type-I
// discrete sine transforms, F_k = sum_{j=1}^{N-1} f_j sin(pi j k / N), for a
// power-of-two N.  The engine transforms two real sequences a, b at once:
//
//   z_j = a_j + i b_j (j = 1..N-1),  z_0 = z_N = 0,  z_{2N-j} = -z_j,
//   Z = FFT_{2N}(z)   (Stockham radix-4, one radix-2 pass if log2 2N is odd),
//   F_k(a) = -Im Z_k / 2,   F_k(b) = Re Z_k / 2,   k = 1..N-1.
//
// The odd extension of a real sequence has a purely imaginary DFT equal to
// -2i times its DST-I, so packing b as the imaginary part puts its transform
// in the real part.  Every output is a plain FFT output: there is no
// recurrence, so the FP32 rounding error grows like log N (a half-length
// transform whose odd outputs come from a running sum, tried first, lost
// accuracy like sqrt N and missed the FP32 tolerance at N >= 1024).
//
// Twiddles come from one FP64-generated table per N, tw[t] = e^{i pi t/N},
// t = 0..2N-1, stored in the working precision.  A CTA holds `lanes`
// complex sequences of length 2N in shared memory (stride 4N + 2 reals,
// which keeps the transposing column loads free of bank conflicts); each is
// worked on by TPR = 2N/(4 NB) threads doing NB radix-4 butterflies per
// pass.  Every pass reads its operands into registers, synchronises and
// writes in place, so one buffer per sequence suffices.
#include <cuda_runtime.h>

#include "qg_internal.cuh"

namespace qg {
namespace {

template <typename T>
struct Cplx {
    T x, y;
};

template <typename T>
__device__ __forceinline__ Cplx<T> ld_c(const T* b, int m) {
    return Cplx<T>{b[2 * m], b[2 * m + 1]};
}
template <typename T>
__device__ __forceinline__ void st_c(T* b, int m, Cplx<T> v) {
    b[2 * m] = v.x;
    b[2 * m + 1] = v.y;
}
// a * conj(w)
template <typename T, typename W>
__device__ __forceinline__ Cplx<T> cmul_conj(Cplx<T> a, W w) {
    return Cplx<T>{a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y};
}

// Per-sequence thread geometry inside a CTA.
struct Geo {
    int N;      // DST length parameter (N - 1 unknowns)
    int L;      // complex FFT length, 2N
    int logL;
    int TPR;    // threads per sequence
    int t;      // thread index within the sequence
    int lane;   // sequence index within the CTA
};

__device__ __forceinline__ Geo make_geo(int N, int NB) {
    Geo g;
    g.N = N;
    g.L = 2 * N;
    g.logL = 31 - __clz(g.L);
    g.TPR = g.L / (4 * NB);
    g.t = threadIdx.x % g.TPR;
    g.lane = threadIdx.x / g.TPR;
    return g;
}

__host__ __device__ constexpr int lane_stride(int N) { return 4 * N + 2; }

// First pass when log2 L is odd: radix 2 with Ns = 1 (no twiddles).
template <typename T, int NB>
__device__ __forceinline__ void fft_pass2_first(T* buf, const Geo& g) {
    constexpr int B = 2 * NB;
    const int half = g.L >> 1;
    Cplx<T> v0[B], v1[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = g.t + b * g.TPR;
        const Cplx<T> a = ld_c(buf, j);
        const Cplx<T> c = ld_c(buf, j + half);
        v0[b] = Cplx<T>{a.x + c.x, a.y + c.y};
        v1[b] = Cplx<T>{a.x - c.x, a.y - c.y};
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = g.t + b * g.TPR;
        st_c(buf, 2 * j, v0[b]);
        st_c(buf, 2 * j + 1, v1[b]);
    }
    __syncthreads();
}

// One radix-4 Stockham pass with sub-transform size Ns (forward, e^{-i}).
// The twiddle of input r is e^{-2 pi i r k/(4 Ns)} = conj(tw[r k N/(2 Ns)]).
template <typename T, int NB>
__device__ __forceinline__ void fft_pass4(T* buf, const Geo& g, int Ns,
                                          const typename Cx<T>::type* tw) {
    const int quarter = g.L >> 2;
    const int tstep = g.N / (2 * Ns);
    Cplx<T> o[NB][4];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = g.t + b * g.TPR;
        const int k = j & (Ns - 1);
        Cplx<T> v0 = ld_c(buf, j);
        Cplx<T> v1 = ld_c(buf, j + quarter);
        Cplx<T> v2 = ld_c(buf, j + 2 * quarter);
        Cplx<T> v3 = ld_c(buf, j + 3 * quarter);
        if (Ns > 1) {
            v1 = cmul_conj(v1, tw[k * tstep]);
            v2 = cmul_conj(v2, tw[2 * k * tstep]);
            v3 = cmul_conj(v3, tw[3 * k * tstep]);
        }
        const Cplx<T> a0{v0.x + v2.x, v0.y + v2.y};
        const Cplx<T> a1{v0.x - v2.x, v0.y - v2.y};
        const Cplx<T> a2{v1.x + v3.x, v1.y + v3.y};
        const Cplx<T> a3{v1.y - v3.y, v3.x - v1.x};   // -i (v1 - v3)
        o[b][0] = Cplx<T>{a0.x + a2.x, a0.y + a2.y};
        o[b][2] = Cplx<T>{a0.x - a2.x, a0.y - a2.y};
        o[b][1] = Cplx<T>{a1.x + a3.x, a1.y + a3.y};
        o[b][3] = Cplx<T>{a1.x - a3.x, a1.y - a3.y};
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int j = g.t + b * g.TPR;
        const int k = j & (Ns - 1);
        const int d = (j - k) * 4 + k;
        st_c(buf, d, o[b][0]);
        st_c(buf, d + Ns, o[b][1]);
        st_c(buf, d + 2 * Ns, o[b][2]);
        st_c(buf, d + 3 * Ns, o[b][3]);
    }
    __syncthreads();
}

// Forward complex FFT of length L in place (buf holds L interleaved complex
// values).  Must be reached by every thread of the CTA.
template <typename T, int NB>
__device__ __forceinline__ void fft_inplace(T* buf, const Geo& g,
                                            const typename Cx<T>::type* tw) {
    int Ns = 1;
    if (g.logL & 1) {
        fft_pass2_first<T, NB>(buf, g);
        Ns = 2;
    }
    for (; Ns < g.L; Ns <<= 2) fft_pass4<T, NB>(buf, g, Ns, tw);
}

// Write z_j = (a_j, b_j) and its odd extension z_{2N-j} = -z_j (j >= 1);
// j = 0 also clears z_N.
template <typename T>
__device__ __forceinline__ void put_pair(T* buf, int N, int j, T a, T b) {
    if (j == 0) {
        buf[0] = T(0);
        buf[1] = T(0);
        buf[2 * N] = T(0);
        buf[2 * N + 1] = T(0);
    } else {
        buf[2 * j] = a;
        buf[2 * j + 1] = b;
        buf[2 * (2 * N - j)] = -a;
        buf[2 * (2 * N - j) + 1] = -b;
    }
}

// Rows kernel: each lane transforms rows r0 = 1 + 2p and r1 = r0 + 1.
template <typename T, int NB>
__global__ void __launch_bounds__(512)
dst_rows_kernel(RowInput<T> in, T* out, int ld, int nrows, int N,
                const typename Cx<T>::type* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geo g = make_geo(N, NB);
    const int lanes = blockDim.x / g.TPR;
    T* buf = reinterpret_cast<T*>(smem_raw) + g.lane * lane_stride(N);
    const int r0 = 1 + 2 * (blockIdx.x * lanes + g.lane);
    const int r1 = r0 + 1;
    const bool v0 = r0 <= nrows, v1 = r1 <= nrows;
    const size_t o0 = (size_t)r0 * ld, o1 = (size_t)r1 * ld;
    for (int j = g.t; j < N; j += g.TPR) {
        T a = T(0), b = T(0);
        if (j > 0) {
            for (int q = 0; q < in.n; ++q) {
                if (v0) a += in.p[q][o0 + j];
                if (v1) b += in.p[q][o1 + j];
            }
        }
        put_pair(buf, N, j, a, b);
    }
    __syncthreads();
    fft_inplace<T, NB>(buf, g, tw);
    T* d0 = out + (size_t)r0 * ld;
    T* d1 = out + (size_t)r1 * ld;
    for (int k = g.t; k < N; k += g.TPR) {
        if (v0) d0[k] = (k == 0) ? T(0) : T(-0.5) * buf[2 * k + 1];
        if (v1) d1[k] = (k == 0) ? T(0) : T(0.5) * buf[2 * k];
    }
}

// Column panel load: c = 2p + part enumerates the 2*lanes sequences of the
// CTA; sequence c comes from plane `src(c)` column `col(c)`.
template <typename T, typename Src>
__device__ __forceinline__ void load_panel(T* base, int N, int lanes, int ld,
                                           Src src) {
    const int nseq = 2 * lanes;
    for (int idx = threadIdx.x; idx < N * nseq; idx += blockDim.x) {
        const int c = idx % nseq, j = idx / nseq;
        const int p = c >> 1, part = c & 1;
        T* buf = base + p * lane_stride(N);
        const T* s = src(c);
        const T v = (j > 0 && s) ? s[(size_t)j * ld] : T(0);
        if (j == 0) {
            buf[part] = T(0);
            buf[2 * N + part] = T(0);
        } else {
            buf[2 * j + part] = v;
            buf[2 * (2 * N - j) + part] = -v;
        }
    }
}

template <typename T, typename Dst>
__device__ __forceinline__ void store_panel(const T* base, int N, int lanes,
                                            int ld, Dst dst) {
    const int nseq = 2 * lanes;
    for (int idx = threadIdx.x; idx < N * nseq; idx += blockDim.x) {
        const int c = idx % nseq, j = idx / nseq;
        if (j == 0) continue;
        T* d = dst(c);
        if (!d) continue;
        const T* buf = base + (c >> 1) * lane_stride(N);
        d[(size_t)j * ld] = (c & 1) ? T(0.5) * buf[2 * j] : T(-0.5) * buf[2 * j + 1];
    }
}

// One-layer column pass: forward DST-I along y of columns col_a = col0+2p
// and col_b = col_a+1, psihat = scale Qhat/(lamx[k] + lamy[l]), inverse.
template <typename T, int NB>
__global__ void __launch_bounds__(512)
dst_cols_solve_kernel(T* __restrict__ data, int ld, int ncols, int N,
                      const typename Cx<T>::type* __restrict__ tw,
                      const T* __restrict__ lamx, const T* __restrict__ lamy,
                      T scale) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geo g = make_geo(N, NB);
    const int lanes = blockDim.x / g.TPR;
    T* base = reinterpret_cast<T*>(smem_raw);
    T* buf = base + g.lane * lane_stride(N);
    const int col0 = 1 + blockIdx.x * 2 * lanes;
    load_panel<T>(base, N, lanes, ld, [&](int c) -> const T* {
        const int col = col0 + c;
        return col <= ncols ? data + col : nullptr;
    });
    __syncthreads();
    fft_inplace<T, NB>(buf, g, tw);
    const int ca = col0 + 2 * g.lane, cb = ca + 1;
    const T lxa = ca <= ncols ? lamx[ca] : T(0);
    const T lxb = cb <= ncols ? lamx[cb] : T(0);
    for (int l = g.t; l < N; l += g.TPR) {
        T a = T(0), b = T(0);
        if (l > 0) {
            const T Fa = T(-0.5) * buf[2 * l + 1];
            const T Fb = T(0.5) * buf[2 * l];
            const T ly = lamy[l];
            a = ca <= ncols ? Fa * (scale / (lxa + ly)) : T(0);
            b = cb <= ncols ? Fb * (scale / (lxb + ly)) : T(0);
        }
        put_pair(buf, N, l, a, b);
    }
    __syncthreads();
    fft_inplace<T, NB>(buf, g, tw);
    store_panel<T>(base, N, lanes, ld, [&](int c) -> T* {
        const int col = col0 + c;
        return col <= ncols ? data + col : nullptr;
    });
}

// Two-layer column pass: lane p holds column col0+p of both planes (layer 1
// as the real part, layer 2 as the imaginary part), so the coupled 2x2
// system of Eqs. isub-1/2 is solved mode by mode inside the lane.
template <typename T, int NB>
__global__ void __launch_bounds__(512)
dst_cols_solve2_kernel(T* __restrict__ d0, T* __restrict__ d1, int ld,
                       int ncols, int N,
                       const typename Cx<T>::type* __restrict__ tw,
                       const T* __restrict__ lamx, const T* __restrict__ lamy,
                       T scale, T Ro, T f1, T f2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geo g = make_geo(N, NB);
    const int lanes = blockDim.x / g.TPR;
    T* base = reinterpret_cast<T*>(smem_raw);
    T* buf = base + g.lane * lane_stride(N);
    const int col0 = 1 + blockIdx.x * lanes;
    load_panel<T>(base, N, lanes, ld, [&](int c) -> const T* {
        const int col = col0 + (c >> 1);
        return col <= ncols ? ((c & 1) ? d1 : d0) + col : nullptr;
    });
    __syncthreads();
    fft_inplace<T, NB>(buf, g, tw);
    const int col = col0 + g.lane;
    const T lx = col <= ncols ? lamx[col] : T(0);
    for (int l = g.t; l < N; l += g.TPR) {
        T p1 = T(0), p2 = T(0);
        if (l > 0 && col <= ncols) {
            const T q1 = T(-0.5) * scale * buf[2 * l + 1];
            const T q2 = T(0.5) * scale * buf[2 * l];
            const T a = Ro * (lx + lamy[l]);
            const T den = a * (a - f1 - f2);
            p1 = (a * q1 - f2 * q1 - f1 * q2) / den;
            p2 = (a * q2 - f2 * q1 - f1 * q2) / den;
        }
        put_pair(buf, N, l, p1, p2);
    }
    __syncthreads();
    fft_inplace<T, NB>(buf, g, tw);
    store_panel<T>(base, N, lanes, ld, [&](int c) -> T* {
        const int cc = col0 + (c >> 1);
        return cc <= ncols ? ((c & 1) ? d1 : d0) + cc : nullptr;
    });
}

template <typename T>
size_t dst_smem(int N, int lanes) {
    return sizeof(T) * (size_t)lanes * lane_stride(N);
}

}  // namespace

// Launch shapes: NB grows until a sequence has at most 256 threads.
static int pick_nb(int N) {
    const int L = 2 * N;
    int nb = 1;
    while (L / (4 * nb) > 256 && nb < 8) nb <<= 1;
    return nb;
}

static constexpr size_t kSmemCap = 200 * 1024;

DstLaunch dst_rows_config(int N, size_t esz) {
    DstLaunch c;
    c.nb = pick_nb(N);
    const int tpr = (2 * N) / (4 * c.nb);
    int lanes = 256 / tpr;
    if (lanes < 1) lanes = 1;
    while (lanes > 1 && esz * (size_t)lanes * lane_stride(N) > 64 * 1024) lanes >>= 1;
    c.lanes = lanes;
    return c;
}

DstLaunch dst_cols_config(int N, size_t esz) {
    DstLaunch c;
    c.nb = pick_nb(N);
    const int tpr = (2 * N) / (4 * c.nb);
    int lanes = 512 / tpr;
    if (lanes < 1) lanes = 1;
    if (lanes > 8) lanes = 8;
    while (lanes > 1 && esz * (size_t)lanes * lane_stride(N) > kSmemCap) lanes >>= 1;
    c.lanes = lanes;
    return c;
}

size_t dst_max_smem() { return kSmemCap; }
size_t dst_lane_bytes(int N, size_t esz) { return esz * (size_t)lane_stride(N); }

template <typename K>
static cudaError_t allow_smem(K k) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmemCap);
}

cudaError_t dst_prepare_kernels() {
    cudaError_t e = cudaSuccess;
#define QG_ALLOW(T, NB)                                                        \
    if (e == cudaSuccess) e = allow_smem(dst_rows_kernel<T, NB>);            \
    if (e == cudaSuccess) e = allow_smem(dst_cols_solve_kernel<T, NB>);      \
    if (e == cudaSuccess) e = allow_smem(dst_cols_solve2_kernel<T, NB>);
    QG_ALLOW(float, 1) QG_ALLOW(float, 2) QG_ALLOW(float, 4) QG_ALLOW(float, 8)
    QG_ALLOW(double, 1) QG_ALLOW(double, 2) QG_ALLOW(double, 4) QG_ALLOW(double, 8)
#undef QG_ALLOW
    return e;
}

template <typename T>
cudaError_t launch_dst_rows(RowInput<T> in, T* out, int ld, int nrows, int N,
                            const typename Cx<T>::type* tw, DstLaunch cfg,
                            cudaStream_t s) {
    const int tpr = (2 * N) / (4 * cfg.nb);
    const dim3 block(tpr * cfg.lanes);
    const int pairs = (nrows + 1) / 2;
    const dim3 grid((pairs + cfg.lanes - 1) / cfg.lanes);
    const size_t sm = dst_smem<T>(N, cfg.lanes);
    switch (cfg.nb) {
        case 1: dst_rows_kernel<T, 1><<<grid, block, sm, s>>>(in, out, ld, nrows, N, tw); break;
        case 2: dst_rows_kernel<T, 2><<<grid, block, sm, s>>>(in, out, ld, nrows, N, tw); break;
        case 4: dst_rows_kernel<T, 4><<<grid, block, sm, s>>>(in, out, ld, nrows, N, tw); break;
        case 8: dst_rows_kernel<T, 8><<<grid, block, sm, s>>>(in, out, ld, nrows, N, tw); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dst_cols_solve(T* data, int ld, int ncols, int N,
                                  const typename Cx<T>::type* tw,
                                  const T* lamx, const T* lamy, T scale,
                                  DstLaunch cfg, cudaStream_t s) {
    const int tpr = (2 * N) / (4 * cfg.nb);
    const dim3 block(tpr * cfg.lanes);
    const int per = 2 * cfg.lanes;
    const dim3 grid((ncols + per - 1) / per);
    const size_t sm = dst_smem<T>(N, cfg.lanes);
    switch (cfg.nb) {
        case 1: dst_cols_solve_kernel<T, 1><<<grid, block, sm, s>>>(data, ld, ncols, N, tw, lamx, lamy, scale); break;
        case 2: dst_cols_solve_kernel<T, 2><<<grid, block, sm, s>>>(data, ld, ncols, N, tw, lamx, lamy, scale); break;
        case 4: dst_cols_solve_kernel<T, 4><<<grid, block, sm, s>>>(data, ld, ncols, N, tw, lamx, lamy, scale); break;
        case 8: dst_cols_solve_kernel<T, 8><<<grid, block, sm, s>>>(data, ld, ncols, N, tw, lamx, lamy, scale); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dst_cols_solve2(T* d0, T* d1, int ld, int ncols, int N,
                                   const typename Cx<T>::type* tw,
                                   const T* lamx, const T* lamy, T scale,
                                   T Ro, T f1, T f2, DstLaunch cfg,
                                   cudaStream_t s) {
    const int tpr = (2 * N) / (4 * cfg.nb);
    const dim3 block(tpr * cfg.lanes);
    const dim3 grid((ncols + cfg.lanes - 1) / cfg.lanes);
    const size_t sm = dst_smem<T>(N, cfg.lanes);
    switch (cfg.nb) {
        case 1: dst_cols_solve2_kernel<T, 1><<<grid, block, sm, s>>>(d0, d1, ld, ncols, N, tw, lamx, lamy, scale, Ro, f1, f2); break;
        case 2: dst_cols_solve2_kernel<T, 2><<<grid, block, sm, s>>>(d0, d1, ld, ncols, N, tw, lamx, lamy, scale, Ro, f1, f2); break;
        case 4: dst_cols_solve2_kernel<T, 4><<<grid, block, sm, s>>>(d0, d1, ld, ncols, N, tw, lamx, lamy, scale, Ro, f1, f2); break;
        case 8: dst_cols_solve2_kernel<T, 8><<<grid, block, sm, s>>>(d0, d1, ld, ncols, N, tw, lamx, lamy, scale, Ro, f1, f2); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

#define QG_INST(T)                                                               \
    template cudaError_t launch_dst_rows<T>(RowInput<T>, T*, int, int, int,       \
                                            const Cx<T>::type*, DstLaunch,        \
                                            cudaStream_t);                        \
    template cudaError_t launch_dst_cols_solve<T>(T*, int, int, int,              \
                                                  const Cx<T>::type*, const T*,   \
                                                  const T*, T, DstLaunch,         \
                                                  cudaStream_t);                  \
    template cudaError_t launch_dst_cols_solve2<T>(T*, T*, int, int, int,         \
                                                   const Cx<T>::type*, const T*,  \
                                                   const T*, T, T, T, T,          \
                                                   DstLaunch, cudaStream_t);
QG_INST(float)
QG_INST(double)
#undef QG_INST

}  // namespace qg
