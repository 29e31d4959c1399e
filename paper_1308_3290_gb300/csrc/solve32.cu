// Elliptic solve of Section 4.3 with a warp-group FFT engine (radix 32).
//
// Same three phases and the same transforms as solve.cu (x pass of the
// right-hand side; y pass with the eigenvalue division of Eq. ialpha or the
// coupled solve of Eqs. isub-1/2; inverse x pass), and the same pairing of
// two real sequences into one complex FFT of length L = 2N of their odd
// extensions (F(a) = -Im Z / 2, F(b) = Re Z / 2).  What differs is the FFT:
//
//   * a pair belongs to a group of G = L/32 threads, and every thread holds
//     32 complex values in registers through each Stockham pass, so a pass
//     is one 32-point DFT per thread between two shared-memory exchanges;
//     L = 1024 takes two radix-32 passes, L = 2048 two and one radix-2 pass;
//   * the exchanges synchronise only the group: __syncwarp when G <= 32, a
//     named barrier of G threads otherwise, so independent pairs never wait
//     for one another (the block-wide barriers between the passes of the
//     shared-memory engine were its main stall);
//   * the odd extension is never stored: the first pass reads z_j or -z_{L-j}
//     from the N stored values;
//   * the twiddles of pass p >= 1 come from a per-pass table laid out
//     [r][k] (k fastest), so a warp reads consecutive entries.
//
// The x pass writes its spectrum transposed with column c = row - 1, so a
// pair's two rows land in one aligned 2-vector; the y pass writes back with
// column k - 1 likewise, and the inverse x pass reads that shift back.
#include <cuda_runtime.h>

#include "dst_engine.cuh"
#include "qg_internal.cuh"

namespace qg {

size_t pass_table_size(int L) {
    int lg = 0;
    while ((1 << lg) < L) ++lg;
    const int np = lg / 5, rem = lg % 5;
    size_t n = 0;
    int ns = 32;
    for (int p = 1; p < np; ++p, ns *= 32) n += (size_t)32 * ns;
    if (rem > 0 && np >= 1) n += (size_t)(1 << rem) * ns;
    return n;
}

void pass_table(int L, double* re, double* im) {
    int lg = 0;
    while ((1 << lg) < L) ++lg;
    const int np = lg / 5, rem = lg % 5;
    const double pi = 3.14159265358979323846;
    size_t o = 0;
    int ns = 32;
    auto block = [&](int R, int Ns) {
        for (int r = 0; r < R; ++r)
            for (int k = 0; k < Ns; ++k) {
                const double a = -2.0 * pi * (double)r * (double)k / ((double)R * (double)Ns);
                re[o] = std::cos(a);
                im[o] = std::sin(a);
                ++o;
            }
    };
    for (int p = 1; p < np; ++p, ns *= 32) block(32, ns);
    if (rem > 0 && np >= 1) block(1 << rem, ns);
}

namespace {

using namespace eng;

constexpr int kT = 256;                 // most threads per CTA
constexpr int kSpin = 1 << 22;
constexpr int kMinLog = 5, kMaxLog = 13;   // L = 32 .. 8192

__host__ __device__ constexpr int px(int m) { return m + (m >> 5); }

template <int LOG>
struct Pl {
    static constexpr int L = 1 << LOG, N = L / 2, G = L / 32;
    static constexpr int NP = LOG / 5, REM = LOG % 5;
    static constexpr int BUF = px(L) + 2;        // padded complex per pair
};

// CTA size: one pair of the longer direction (at least a warp), so that the
// few pairs of a small elliptic grid spread over many SMs.
__host__ __device__ constexpr int cta_threads(int lgx, int lgy) {
    const int g = ((1 << (lgx > lgy ? lgx : lgy)) / 32);
    return g < 32 ? 32 : g;
}
__host__ __device__ constexpr int buf_cplx(int lg, int threads) {
    return (threads / ((1 << lg) / 32)) * (px(1 << lg) + 2);
}

// Group barrier: the G threads of one pair.
struct Sync {
    int id, n;
    __device__ __forceinline__ void sync() const {
        if (n <= 32) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
    }
};

template <typename T>
__device__ __forceinline__ Cplx<T> ldp(const CT<T>* b, int m) {
    const CT<T> v = b[px(m)];
    return Cplx<T>{v.x, v.y};
}
template <typename T>
__device__ __forceinline__ void stp(CT<T>* b, int m, Cplx<T> v) {
    CT<T> w;
    w.x = v.x;
    w.y = v.y;
    b[px(m)] = w;
}

// e^{-2 pi i e/32} = (c, -s) for 0 <= e < 24, from the first-quadrant values.
template <typename T>
__device__ __forceinline__ void w32(int e, T& c, T& s) {
    T c0 = T(1), s0 = T(0);
    switch (e & 7) {
        case 1: c0 = T(0.9807852804032304491261822); s0 = T(0.1950903220161282678482849); break;
        case 2: c0 = T(0.9238795325112867561281832); s0 = T(0.3826834323650897717284600); break;
        case 3: c0 = T(0.8314696123025452370787884); s0 = T(0.5555702330196022247428308); break;
        case 4: c0 = T(0.7071067811865475244008444); s0 = T(0.7071067811865475244008444); break;
        case 5: c0 = T(0.5555702330196022247428308); s0 = T(0.8314696123025452370787884); break;
        case 6: c0 = T(0.3826834323650897717284600); s0 = T(0.9238795325112867561281832); break;
        case 7: c0 = T(0.1950903220161282678482849); s0 = T(0.9807852804032304491261822); break;
        default: break;
    }
    switch (e >> 3) {   // rotate by quarter turns
        case 0: c = c0; s = s0; break;
        case 1: c = -s0; s = c0; break;
        default: c = -c0; s = -s0; break;
    }
}

template <typename T>
__device__ __forceinline__ Cplx<T> tw_mul(Cplx<T> v, int e) {
    if (e == 0) return v;
    if (e == 8) return cmi(v);
    if (e == 16) return Cplx<T>{-v.x, -v.y};
    T c, s;
    w32<T>(e, c, s);
    return Cplx<T>{v.x * c + v.y * s, v.y * c - v.x * s};
}

// 8-point DFT, natural order: n = m1 + 2 m2, two 4-point DFTs, twiddles, 2-point.
template <typename T>
__device__ __forceinline__ void dft8n(Cplx<T> (&e)[8]) {
    dft4(e[0], e[2], e[4], e[6]);
    dft4(e[1], e[3], e[5], e[7]);
    const T r2 = T(0.7071067811865475244008444);
    e[3] = cmul(e[3], r2, -r2);
    e[5] = cmi(e[5]);
    e[7] = cmul(e[7], -r2, -r2);
    Cplx<T> o[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        o[k] = cadd(e[2 * k], e[2 * k + 1]);
        o[k + 4] = csub(e[2 * k], e[2 * k + 1]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) e[k] = o[k];
}

// 32-point DFT in place, natural order: n = n1 + 4 n2, k = k2 + 8 k1.
template <typename T>
__device__ __forceinline__ void dft32(Cplx<T> (&v)[32]) {
    Cplx<T> y[4][8];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) y[n1][n2] = v[n1 + 4 * n2];
        dft8n<T>(y[n1]);
    }
#pragma unroll
    for (int n1 = 1; n1 < 4; ++n1)
#pragma unroll
        for (int k2 = 1; k2 < 8; ++k2) y[n1][k2] = tw_mul<T>(y[n1][k2], n1 * k2);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
        dft4(y[0][k2], y[1][k2], y[2][k2], y[3][k2]);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) v[k2 + 8 * k1] = y[k1][k2];
    }
}

// Element m = t + r G of the odd extension of z (stored at 0..N-1, z_0 = 0).
template <typename T, int LOG>
__device__ __forceinline__ Cplx<T> first_read(const CT<T>* cb, int t, int r) {
    using P = Pl<LOG>;
    if (r < 16) return ldp<T>(cb, t + r * P::G);
    if (r == 16) {
        if (t == 0) return Cplx<T>{T(0), T(0)};
        const Cplx<T> z = ldp<T>(cb, P::N - t);
        return Cplx<T>{-z.x, -z.y};
    }
    const Cplx<T> z = ldp<T>(cb, (32 - r) * P::G - t);
    return Cplx<T>{-z.x, -z.y};
}

// One Stockham pass of radix R with sub-transform size NS: every thread does
// 32/R butterflies j = t + b G; input j + r L/R, output (j - k) R + k + r NS.
template <typename T, int LOG, int R, int NS, bool FIRST>
__device__ __forceinline__ void pass(CT<T>* cb, int t, const CT<T>* __restrict__ tw,
                                     const Sync& sy) {
    using P = Pl<LOG>;
    constexpr int B = 32 / R, STRIDE = P::L / R;
    Cplx<T> v[B][R];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + b * P::G;
        const int k = j & (NS - 1);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if constexpr (FIRST) v[b][r] = first_read<T, LOG>(cb, t, r);
            else v[b][r] = ldp<T>(cb, j + r * STRIDE);
        }
        if constexpr (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const CT<T> w = __ldg(tw + r * NS + k);
                v[b][r] = cmul(v[b][r], w.x, w.y);
            }
        }
        if constexpr (R == 32) dft32<T>(v[b]);
        else dft<T, R>(v[b]);
    }
    sy.sync();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + b * P::G;
        const int k = j & (NS - 1);
        const int d = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if constexpr (R == 32) stp<T>(cb, d + r * NS, v[b][r]);
            else stp<T>(cb, d + r * NS, v[b][out_slot<R>(r)]);
        }
    }
    sy.sync();
}

// Forward FFT of length L of the odd extension of cb[0..N) in place; the
// result Z_k is at cb[px(k)], k = 0..L-1.  Starts and ends with a group sync.
template <typename T, int LOG>
__device__ __forceinline__ void fft(CT<T>* cb, int t, const CT<T>* tw, const Sync& sy) {
    using P = Pl<LOG>;
    sy.sync();
    pass<T, LOG, 32, 1, true>(cb, t, tw, sy);
    if constexpr (P::NP >= 2) pass<T, LOG, 32, 32, false>(cb, t, tw, sy);
    if constexpr (P::REM > 0)
        pass<T, LOG, (1 << P::REM), (P::NP >= 2 ? 1024 : 32), false>(
            cb, t, tw + (P::NP >= 2 ? 1024 : 0), sy);
}

template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&o)[4]);
template <>
__device__ __forceinline__ void ld4<float>(const float* p, float (&o)[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double* p, double (&o)[4]) {
    const double2 v0 = __ldg(reinterpret_cast<const double2*>(p));
    const double2 v1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
    o[0] = v0.x; o[1] = v0.y; o[2] = v1.x; o[3] = v1.y;
}

template <typename T>
__device__ __forceinline__ void st2(T* p, T a, T b) {
    CT<T> v;
    v.x = a;
    v.y = b;
    *reinterpret_cast<CT<T>*>(p) = v;
}

// Row r of the right-hand side, elements c0..c0+3: plane 0, plus plane 2 on
// rows r % part_py == 0, plus planes 1 and 3 at the column c0 when
// c0 % part_px == 0 (part_px is a multiple of 4).
template <typename T>
__device__ __forceinline__ void rhs4(const SolveParams<T>& P, int layer, int r, int c0,
                                     T (&o)[4]) {
    const size_t off = (size_t)r * P.ld + c0;
    ld4<T>(P.in[layer][0] + off, o);
    if (P.nin > 1) {
        const bool ry = r % P.part_py == 0;
        if (ry) {
            T e[4];
            ld4<T>(P.in[layer][2] + off, e);
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] += e[q];
        }
        if (c0 % P.part_px == 0) {
            o[0] += __ldg(P.in[layer][1] + off);
            if (ry) o[0] += __ldg(P.in[layer][3] + off);
        }
    }
}

// Phase 1: pairs of rows (ra, ra + 1) -> DST over x -> tr[k][ra - 1 .. ra].
template <typename T, int LOG>
__device__ void rows_fwd(const SolveParams<T>& P, CT<T>* bufs) {
    using Q = Pl<LOG>;
    const int grp = threadIdx.x / Q::G, t = threadIdx.x % Q::G;
    CT<T>* cb = bufs + grp * Q::BUF;
    const Sync sy{1 + grp, Q::G};
    const int nrows = P.my - 1;
    const int ppl = (nrows + 1) / 2;
    const int npairs = ppl * P.layers;
    const int per = blockDim.x / Q::G;
    const int nslots = (npairs + per - 1) / per;
    for (int slot = blockIdx.x; slot < nslots; slot += gridDim.x) {
        const int pair = slot * per + grp;
        const bool pv = pair < npairs;
        const int layer = pv ? pair / ppl : 0;
        const int ra = 1 + 2 * (pv ? pair % ppl : 0), rb = ra + 1;
        const bool vb = pv && rb <= nrows;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c0 = 4 * (t + i * Q::G);
            T a[4] = {T(0), T(0), T(0), T(0)}, b[4] = {T(0), T(0), T(0), T(0)};
            if (pv) rhs4<T>(P, layer, ra, c0, a);
            if (vb) rhs4<T>(P, layer, rb, c0, b);
#pragma unroll
            for (int q = 0; q < 4; ++q) stp<T>(cb, c0 + q, Cplx<T>{a[q], b[q]});
        }
        if (t == 0) stp<T>(cb, 0, Cplx<T>{T(0), T(0)});
        fft<T, LOG>(cb, t, P.ptx, sy);
        if (pv) {
            T* tr = P.tr[layer] + (ra - 1);
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
                const int k = t + i * Q::G;
                if (k == 0) continue;
                const CT<T> z = cb[px(k)];
                if (vb) st2<T>(tr + (size_t)k * P.ld_tr, T(-0.5) * z.y, T(0.5) * z.x);
                else tr[(size_t)k * P.ld_tr] = T(-0.5) * z.y;
            }
        }
        sy.sync();
    }
}

// Phase 2: pairs of x-modes -> DST over y, mode-space solve, DST over y ->
// work[j][k - 1].  OPY 1: modes (ka, ka + 1) of one layer; OPY 2: mode k of
// both layers (the coupled 2x2 solve).
template <typename T, int LOG, int OPY>
__device__ void cols_solve(const SolveParams<T>& P, CT<T>* bufs) {
    using Q = Pl<LOG>;
    const int grp = threadIdx.x / Q::G, t = threadIdx.x % Q::G;
    CT<T>* cb = bufs + grp * Q::BUF;
    const Sync sy{1 + grp, Q::G};
    const int ncols = P.mx - 1;
    const int npairs = OPY == 2 ? ncols : (ncols + 1) / 2;
    const int per = blockDim.x / Q::G;
    const int nslots = (npairs + per - 1) / per;
    for (int slot = blockIdx.x; slot < nslots; slot += gridDim.x) {
        const int pair = slot * per + grp;
        const bool pv = pair < npairs;
        int ka, kb;
        const T *sa, *sb;
        if (OPY == 2) {
            ka = kb = 1 + (pv ? pair : 0);
            sa = P.tr[0] + (size_t)ka * P.ld_tr;
            sb = P.tr[1] + (size_t)kb * P.ld_tr;
        } else {
            ka = 1 + 2 * (pv ? pair : 0);
            kb = ka + 1;
            sa = P.tr[0] + (size_t)ka * P.ld_tr;
            sb = P.tr[0] + (size_t)kb * P.ld_tr;
        }
        const bool va = pv, vb = pv && (OPY == 2 || kb <= ncols);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c0 = 4 * (t + i * Q::G);
            T a[4] = {T(0), T(0), T(0), T(0)}, b[4] = {T(0), T(0), T(0), T(0)};
            if (va) ld4<T>(sa + c0, a);
            if (vb) ld4<T>(sb + c0, b);
#pragma unroll
            for (int q = 0; q < 4; ++q) stp<T>(cb, c0 + 1 + q, Cplx<T>{a[q], b[q]});
        }
        if (t == 0) stp<T>(cb, 0, Cplx<T>{T(0), T(0)});
        fft<T, LOG>(cb, t, P.pty, sy);
        const T lxa = __ldg(P.lamx + ka), lxb = __ldg(P.lamx + kb);
#pragma unroll 4
        for (int i = 0; i < 16; ++i) {
            const int l = t + i * Q::G;
            const Cplx<T> z = ldp<T>(cb, l);
            const T Fa = T(-0.5) * z.y, Fb = T(0.5) * z.x;
            T a = T(0), b = T(0);
            if (l > 0 && pv) {
                const T ly = __ldg(P.lamy + l);
                if (OPY == 1) {
                    a = Fa * (P.scale / (lxa + ly));
                    if (vb) b = Fb * (P.scale / (lxb + ly));
                } else {
                    const T q1 = P.scale * Fa, q2 = P.scale * Fb;
                    const T al = P.Ro * (lxa + ly);
                    const T den = al * (al - P.f1 - P.f2);
                    a = (al * q1 - P.f2 * q1 - P.f1 * q2) / den;
                    b = (al * q2 - P.f2 * q1 - P.f1 * q2) / den;
                }
            }
            stp<T>(cb, l, Cplx<T>{a, b});
        }
        fft<T, LOG>(cb, t, P.pty, sy);
        if (pv) {
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
                const int j = t + i * Q::G;
                if (j == 0) continue;
                const CT<T> z = cb[px(j)];
                const T ga = T(-0.5) * z.y, gb = T(0.5) * z.x;
                if (OPY == 2) {
                    P.work[0][(size_t)j * P.ld + ka - 1] = ga;
                    P.work[1][(size_t)j * P.ld + kb - 1] = gb;
                } else if (vb) {
                    st2<T>(P.work[0] + (size_t)j * P.ld + ka - 1, ga, gb);
                } else {
                    P.work[0][(size_t)j * P.ld + ka - 1] = ga;
                }
            }
        }
        sy.sync();
    }
}

// Phase 3: pairs of rows of work (element k at column k - 1) -> DST over x
// -> out[r][k], k = 0..mx-1 (k = 0 is the wall).
template <typename T, int LOG>
__device__ void rows_inv(const SolveParams<T>& P, CT<T>* bufs) {
    using Q = Pl<LOG>;
    const int grp = threadIdx.x / Q::G, t = threadIdx.x % Q::G;
    CT<T>* cb = bufs + grp * Q::BUF;
    const Sync sy{1 + grp, Q::G};
    const int nrows = P.my - 1;
    const int ppl = (nrows + 1) / 2;
    const int npairs = ppl * P.layers;
    const int per = blockDim.x / Q::G;
    const int nslots = (npairs + per - 1) / per;
    for (int slot = blockIdx.x; slot < nslots; slot += gridDim.x) {
        const int pair = slot * per + grp;
        const bool pv = pair < npairs;
        const int layer = pv ? pair / ppl : 0;
        const int ra = 1 + 2 * (pv ? pair % ppl : 0), rb = ra + 1;
        const bool vb = pv && rb <= nrows;
        const T* wa = P.work[layer] + (size_t)ra * P.ld;
        const T* wb = P.work[layer] + (size_t)rb * P.ld;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c0 = 4 * (t + i * Q::G);
            T a[4] = {T(0), T(0), T(0), T(0)}, b[4] = {T(0), T(0), T(0), T(0)};
            if (pv) ld4<T>(wa + c0, a);
            if (vb) ld4<T>(wb + c0, b);
#pragma unroll
            for (int q = 0; q < 4; ++q) stp<T>(cb, c0 + 1 + q, Cplx<T>{a[q], b[q]});
        }
        if (t == 0) stp<T>(cb, 0, Cplx<T>{T(0), T(0)});
        fft<T, LOG>(cb, t, P.ptx, sy);
        if (pv) {
            T* oa = P.out[layer] + (size_t)ra * P.ld;
            T* ob = P.out[layer] + (size_t)rb * P.ld;
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
                const int k = t + i * Q::G;
                const CT<T> z = cb[px(k)];
                oa[k] = k == 0 ? T(0) : T(-0.5) * z.y;
                if (vb) ob[k] = k == 0 ? T(0) : T(0.5) * z.x;
            }
        }
        sy.sync();
    }
}

// Run phase F for the FFT length 2^lg (5 <= lg <= 13).
#define QG_CASES(F, ...)                                  \
    switch (lg) {                                         \
        case 5: F<T, 5, ##__VA_ARGS__>(P, bufs); break;   \
        case 6: F<T, 6, ##__VA_ARGS__>(P, bufs); break;   \
        case 7: F<T, 7, ##__VA_ARGS__>(P, bufs); break;   \
        case 8: F<T, 8, ##__VA_ARGS__>(P, bufs); break;   \
        case 9: F<T, 9, ##__VA_ARGS__>(P, bufs); break;   \
        case 10: F<T, 10, ##__VA_ARGS__>(P, bufs); break; \
        case 11: F<T, 11, ##__VA_ARGS__>(P, bufs); break; \
        case 12: F<T, 12, ##__VA_ARGS__>(P, bufs); break; \
        case 13: F<T, 13, ##__VA_ARGS__>(P, bufs); break; \
        default: break;                                   \
    }

template <typename T, int OPY>
__global__ void __launch_bounds__(kT, sizeof(T) == 4 ? 2 : 1) solve32_kernel(SolveParams<T> P, int lgx, int lgy) {
    extern __shared__ __align__(16) unsigned char smem[];
    CT<T>* bufs = reinterpret_cast<CT<T>*>(smem);
    pdl_wait();
    pdl_trigger();   // the next fine stage may start staging its own inputs
    const bool all = P.split == 0;
    if (all || P.phase == 0) {
        const int lg = lgx;
        QG_CASES(rows_fwd)
    }
    if (all && !grid_sync(P.bar, P.bar_extra, kSpin)) {
        if (threadIdx.x == 0) atomicExch(P.err, 1);
        return;
    }
    if (all || P.phase == 1) {
        const int lg = lgy;
        QG_CASES(cols_solve, OPY)
    }
    if (all && !grid_sync(P.bar, P.bar_extra, kSpin)) {
        if (threadIdx.x == 0) atomicExch(P.err, 1);
        return;
    }
    if (all || P.phase == 2) {
        const int lg = lgx;
        QG_CASES(rows_inv)
    }
}

int log2i(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

template <typename T, int OPY>
cudaError_t launch32(const SolveParams<T>& P, cudaStream_t s) {
    auto k = solve32_kernel<T, OPY>;
    const size_t sm = solve32_smem_bytes(P.mx, P.my, sizeof(T));
    const int lgx = log2i(2 * P.mx), lgy = log2i(2 * P.my);
    const int threads = cta_threads(lgx, lgy);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, threads, sm)) != cudaSuccess)
        return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    auto slots = [threads](int lg, int npairs) {
        const int pairs = threads / ((1 << lg) / 32);
        return (npairs + pairs - 1) / pairs;
    };
    const int rows = (P.my / 2) * P.layers;
    const int cols = OPY == 2 ? P.mx - 1 : P.mx / 2;
    int want = slots(lgx, rows);
    if (slots(lgy, cols) > want) want = slots(lgy, cols);
    int grid = per * nsm;
    if (want < grid) grid = want;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    if (!P.split) {
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k, P, lgx, lgy);
    }
    SolveParams<T> Q = P;
    for (int ph = 0; ph < 3; ++ph) {
        Q.phase = ph;
        if ((e = cudaLaunchKernelEx(&cfg, k, Q, lgx, lgy)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

bool solve32_supports(int mx, int my) {
    const int lx = log2i(2 * mx), ly = log2i(2 * my);
    return is_pow2(mx) && is_pow2(my) && lx >= kMinLog && lx <= kMaxLog && ly >= kMinLog &&
           ly <= kMaxLog;
}

size_t solve32_smem_bytes(int mx, int my, size_t esz) {
    const int lx = log2i(2 * mx), ly = log2i(2 * my), th = cta_threads(lx, ly);
    const int a = buf_cplx(lx, th), b = buf_cplx(ly, th);
    return (size_t)(a > b ? a : b) * 2 * esz;
}

template <typename T>
cudaError_t launch_solve32(const SolveParams<T>& P, cudaStream_t s) {
    if (!solve32_supports(P.mx, P.my) || !P.ptx || !P.pty) return cudaErrorInvalidValue;
    return P.layers == 2 ? launch32<T, 2>(P, s) : launch32<T, 1>(P, s);
}

template cudaError_t launch_solve32<float>(const SolveParams<float>&, cudaStream_t);
template cudaError_t launch_solve32<double>(const SolveParams<double>&, cudaStream_t);

}  // namespace qg
