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

#include <cmath>
#include <cstdlib>

#include "bounds.cuh"
#include "dst_engine.cuh"
#include "qg_internal.cuh"

namespace qg {

size_t pass_table_size(int L, int rad) {
    int lg = 0, lr = 0;
    while ((1 << lg) < L) ++lg;
    while ((1 << lr) < rad) ++lr;
    const int np = lg / lr, rem = lg % lr;
    size_t n = 0;
    int ns = rad;
    for (int p = 1; p < np; ++p, ns *= rad) n += (size_t)rad * ns;
    if (rem > 0 && np >= 1) n += (size_t)(1 << rem) * ns;
    return n;
}

void pass_table(int L, int rad, double* re, double* im) {
    int lg = 0, lr = 0;
    while ((1 << lg) < L) ++lg;
    while ((1 << lr) < rad) ++lr;
    const int np = lg / lr, rem = lg % lr;
    const double pi = 3.14159265358979323846;
    size_t o = 0;
    int ns = rad;
    auto block = [&](int R, int Ns) {
        for (int r = 0; r < R; ++r)
            for (int k = 0; k < Ns; ++k) {
                const double a = -2.0 * pi * (double)r * (double)k / ((double)R * (double)Ns);
                re[o] = std::cos(a);
                im[o] = std::sin(a);
                ++o;
            }
    };
    for (int p = 1; p < np; ++p, ns *= rad) block(rad, ns);
    if (rem > 0 && np >= 1) block(1 << rem, ns);
}

namespace {

using namespace eng;

// most threads per CTA: 512 for FP32 with 16 values per thread (a pair of
// length-8192 sequences in one group: 2 N = 8192 for the full 2048 x 4096
// grid), else 256
__host__ __device__ constexpr int max_cta(int rad, int esz) {
    return (rad == 16 && esz == 4) ? 512 : 256;
}
constexpr int kSpin = 1 << 22;

__host__ __device__ constexpr int px(int m) { return m + (m >> 4); }

// Geometry of one FFT length L = 2^lg with RAD values per thread (RAD = 32
// or 16): N = L/2, G = L/RAD threads per pair, np radix-RAD passes and a
// remainder pass of radix 2^rem (rem = 0: none).
struct Geo32 {
    int L, N, G, np, rem, buf;
};
__host__ __device__ inline int log2c(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}
__host__ __device__ inline Geo32 geo32(int lg, int rad) {
    Geo32 g;
    const int lr = log2c(rad);
    g.L = 1 << lg;
    g.N = g.L / 2;
    g.G = g.L / rad;
    g.np = lg / lr;
    g.rem = lg % lr;
    g.buf = px(g.L) + 2;    // padded complex per pair
    return g;
}

// CTA size: at least one pair group of the longer direction.
__host__ __device__ inline int cta_threads(int lgx, int lgy, int rad, int least) {
    const int g = (1 << (lgx > lgy ? lgx : lgy)) / rad;
    return g < least ? least : g;
}
// two buffers per pair (the passes alternate between them)
__host__ __device__ inline int buf_cplx(int lg, int rad, int threads) {
    const Geo32 g = geo32(lg, rad);
    return (threads / g.G) * 2 * g.buf;
}

// Group barrier: the G threads of one pair.
struct Sync {
    int id, n;
    __device__ __forceinline__ void sync() const {
        if (n <= 32) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
    }
};

// element m of a pair buffer of `lim` complex entries (lim is only read by
// bounds-checked builds)
template <typename T>
__device__ __forceinline__ Cplx<T> ldp(const CT<T>* b, int m, int lim) {
    (void)lim;
    if (!QG_IN(px(m), lim, 21)) return Cplx<T>{T(0), T(0)};
    const CT<T> v = b[px(m)];
    return Cplx<T>{v.x, v.y};
}
template <typename T>
__device__ __forceinline__ void stp(CT<T>* b, int m, Cplx<T> v, int lim) {
    (void)lim;
    if (!QG_IN(px(m), lim, 22)) return;
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

// One radix-RAD Stockham pass from buffer `in` to buffer `out` (one
// RAD-point DFT per thread, butterfly j = t): input j + r G, twiddle table
// entry r NS + k (k = j mod NS), output (j - k) RAD + k + r NS.  The first
// pass (NS = 1) reads the odd extension of the stored z_0..z_{N-1}: element
// m = t + r G is z_m (r < RAD/2), 0 (m = N), or -z_{L-m}.  The two buffers
// alternate, so one group sync after the stores orders both this pass's
// reads before the next pass's writes and its writes before the next reads.
template <typename T, int RAD>
__device__ __forceinline__ void passW(const CT<T>* in, CT<T>* out, int t, const Geo32& g, int NS,
                                      bool first, const CT<T>* __restrict__ tw, const Sync& sy) {
    constexpr int H = RAD / 2;
    const int k = t & (NS - 1);
    Cplx<T> v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) {
        if (!first) {
            v[r] = ldp<T>(in, t + r * g.G, g.buf);
        } else if (r < H) {
            v[r] = ldp<T>(in, t + r * g.G, g.buf);
        } else {
            const int m = r == H ? g.N - t : (RAD - r) * g.G - t;
            const Cplx<T> z = (r == H && t == 0) ? Cplx<T>{T(0), T(0)} : ldp<T>(in, m, g.buf);
            v[r] = Cplx<T>{-z.x, -z.y};
        }
    }
    if (!first) {
        if constexpr (RAD == 8) {
            // w^1 and w^4 from the table, the other powers as products (at
            // most two roundings deep): 2 shared-memory loads instead of 7
            const CT<T> a = tw[NS + k], b = tw[4 * NS + k];
            const Cplx<T> w1{a.x, a.y}, w4{b.x, b.y};
            const Cplx<T> w2 = cmul(w1, w1.x, w1.y);
            const Cplx<T> w3 = cmul(w2, w1.x, w1.y);
            const Cplx<T> w5 = cmul(w4, w1.x, w1.y);
            const Cplx<T> w6 = cmul(w4, w2.x, w2.y);
            const Cplx<T> w7 = cmul(w4, w3.x, w3.y);
            v[1] = cmul(v[1], w1.x, w1.y);
            v[2] = cmul(v[2], w2.x, w2.y);
            v[3] = cmul(v[3], w3.x, w3.y);
            v[4] = cmul(v[4], w4.x, w4.y);
            v[5] = cmul(v[5], w5.x, w5.y);
            v[6] = cmul(v[6], w6.x, w6.y);
            v[7] = cmul(v[7], w7.x, w7.y);
        } else {
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                const CT<T> w = tw[r * NS + k];
                v[r] = cmul(v[r], w.x, w.y);
            }
        }
    }
    if constexpr (RAD == 32) dft32<T>(v);
    else dft<T, RAD>(v);
    const int d = (t - k) * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) {
        if constexpr (RAD == 32) stp<T>(out, d + r * NS, v[r], g.buf);
        else stp<T>(out, d + r * NS, v[out_slot<RAD>(r)], g.buf);
    }
    sy.sync();
}

// The remainder pass, radix R < RAD: RAD/R butterflies j = t + b G per
// thread.  Inlined for RAD = 8; out of line for RAD = 16 and 32 (inlined
// next to their full-radix passes, their registers spill).
template <typename T, int R, int RAD>
__device__ __forceinline__ void passR_body(const CT<T>* in, CT<T>* out, int t, Geo32 g, int NS,
                                          const CT<T>* __restrict__ tw, Sync sy) {
    constexpr int B = RAD / R;
    const int stride = g.L / R;
    Cplx<T> v[B][R];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + b * g.G;
        const int k = j & (NS - 1);
#pragma unroll
        for (int r = 0; r < R; ++r) v[b][r] = ldp<T>(in, j + r * stride, g.buf);
#pragma unroll
        for (int r = 1; r < R; ++r) {
            const CT<T> w = tw[r * NS + k];
            v[b][r] = cmul(v[b][r], w.x, w.y);
        }
        dft<T, R>(v[b]);
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + b * g.G;
        const int k = j & (NS - 1);
        const int d = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) stp<T>(out, d + r * NS, v[b][out_slot<R>(r)], g.buf);
    }
    sy.sync();
}

template <typename T, int R, int RAD>
__device__ __noinline__ void passR_call(const CT<T>* in, CT<T>* out, int t, Geo32 g, int NS,
                                        const CT<T>* __restrict__ tw, Sync sy) {
    passR_body<T, R, RAD>(in, out, t, g, NS, tw, sy);
}

template <typename T, int R, int RAD>
__device__ __forceinline__ void passR(const CT<T>* in, CT<T>* out, int t, const Geo32& g, int NS,
                                      const CT<T>* __restrict__ tw, const Sync& sy) {
    if constexpr (RAD <= 8) passR_body<T, R, RAD>(in, out, t, g, NS, tw, sy);
    else passR_call<T, R, RAD>(in, out, t, g, NS, tw, sy);
}

// Forward FFT of length L of the odd extension of a[0..N); the passes
// alternate between a and b, and the result Z_k, k = 0..L-1, is at
// [px(k)] of the buffer returned.  Starts and ends with a group sync.
template <typename T, int RAD>
__device__ __forceinline__ CT<T>* fft_rt(CT<T>* a, CT<T>* b, int t, const Geo32& g,
                                         const CT<T>* tw, const Sync& sy) {
    sy.sync();
    int ns = 1, off = 0;
#pragma unroll 1
    for (int p = 0; p < g.np; ++p) {
        passW<T, RAD>(a, b, t, g, ns, p == 0, tw + off, sy);
        CT<T>* c = a;
        a = b;
        b = c;
        if (p > 0) off += RAD * ns;
        ns *= RAD;
    }
    if (g.rem > 0) {
        const CT<T>* tr = tw + off;
        switch (g.rem) {
            case 1: passR<T, 2, RAD>(a, b, t, g, ns, tr, sy); break;
            case 2: passR<T, 4, RAD>(a, b, t, g, ns, tr, sy); break;
            case 3:
                if constexpr (RAD > 8) passR<T, 8, RAD>(a, b, t, g, ns, tr, sy);
                break;
            default:
                if constexpr (RAD == 32) passR<T, 16, RAD>(a, b, t, g, ns, tr, sy);
                break;
        }
        return b;
    }
    return a;
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

// four consecutive values: one 16-byte store (FP32) where p is 16-byte
// aligned, else two 8-byte stores; FP64 two 16-byte stores
template <typename T>
__device__ __forceinline__ void st4(T* p, T a, T b, T c, T d) {
    if constexpr (sizeof(T) == 4) {
        if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
            *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
            return;
        }
    }
    st2<T>(p, a, b);
    st2<T>(p + 2, c, d);
}

// Row r of the right-hand side, elements c0..c0+3: plane 0, plus plane 2 on
// rows r % part_py == 0, plus planes 1 and 3 at the column c0 when
// c0 % part_px == 0 (part_px is a multiple of 4).
template <typename T>
__device__ __forceinline__ void rhs4(const SolveParams<T>& P, int layer, int r, int c0,
                                     T (&o)[4]) {
    const size_t off = (size_t)r * P.ld + c0;
    if (!QG_IN(off + 3, (long long)(P.my + 1) * P.ld, 23)) {
        o[0] = o[1] = o[2] = o[3] = T(0);
        return;
    }
    ld4<T>(P.in[layer][0] + off, o);
    if (P.nin > 1) {
        const bool ry = (r & (P.part_py - 1)) == 0;
        if (ry) {
            T e[4];
            ld4<T>(P.in[layer][2] + off, e);
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] += e[q];
        }
        if ((c0 & (P.part_px - 1)) == 0) {
            o[0] += __ldg(P.in[layer][1] + off);
            if (ry) o[0] += __ldg(P.in[layer][3] + off);
        }
    }
}

// The sequence pair `pair` of phase ph (0: rows of the right-hand side,
// 1: x-modes, 2: rows of work) and where its two sequences live.
struct PairAt {
    bool va, vb;
    int layer;    // phases 0, 2
    int ra, rb;   // rows (phases 0, 2) or x-modes (phase 1)
};

template <typename T, int OPY>
__device__ __forceinline__ PairAt pair_at(const SolveParams<T>& P, int ph, int pair, int npairs) {
    PairAt a;
    const bool pv = pair < npairs;
    if (ph == 1) {
        const int ncols = P.mx - 1;
        a.layer = 0;
        if (OPY == 2) {
            a.ra = a.rb = 1 + (pv ? pair : 0);
        } else {
            a.ra = 1 + 2 * (pv ? pair : 0);
            a.rb = a.ra + 1;
        }
        a.va = pv;
        a.vb = pv && (OPY == 2 || a.rb <= ncols);
    } else {
        const int nrows = P.my - 1, ppl = (nrows + 1) / 2;
        if (OPY == 1) {   // one layer: pairs < ppl, no division
            a.layer = 0;
            a.ra = 1 + 2 * (pv ? pair : 0);
        } else {
            a.layer = pv ? pair / ppl : 0;
            a.ra = 1 + 2 * (pv ? pair % ppl : 0);
        }
        a.rb = a.ra + 1;
        a.va = pv;
        a.vb = pv && a.rb <= nrows;
    }
    return a;
}

// Stage the pair's input z_j = (a_j, b_j), j = 0..N-1, into cb (z_0 = 0).
//   phase 0: rows of the right-hand side (sum of the partial planes);
//   phase 1: rows ka, kb of tr (element j at column j - 1);
//   phase 2: rows of work (element j at column j - 1).
template <typename T, int OPY, int RAD>
__device__ __forceinline__ void load_pair(const SolveParams<T>& P, int ph, const PairAt& a,
                                          const Geo32& g, CT<T>* cb, int t) {
    const T *sa = nullptr, *sb = nullptr;
    if (ph == 1) {
        sa = P.tr[0] + (size_t)a.ra * P.ld_tr;
        sb = P.tr[OPY == 2 ? 1 : 0] + (size_t)a.rb * P.ld_tr;
    } else if (ph == 2) {
        sa = P.work[a.layer] + (size_t)a.ra * P.ld;
        sb = P.work[a.layer] + (size_t)a.rb * P.ld;
    }
    const int shift = ph == 0 ? 0 : 1;
#pragma unroll
    for (int i = 0; i < RAD / 8; ++i) {    // N = (RAD/2) G values, 4 per step
        const int c0 = 4 * (t + i * g.G);
        T x[4] = {T(0), T(0), T(0), T(0)}, y[4] = {T(0), T(0), T(0), T(0)};
        if (ph == 0) {
            if (a.va) rhs4<T>(P, a.layer, a.ra, c0, x);
            if (a.vb) rhs4<T>(P, a.layer, a.rb, c0, y);
        } else {
            // rows of tr (mx + 1 rows of pitch ld_tr) or of work (my + 1 of ld)
            const long long n = ph == 1 ? (long long)(P.mx + 1) * P.ld_tr
                                        : (long long)(P.my + 1) * P.ld;
            const long long pitch = ph == 1 ? P.ld_tr : P.ld;
            if (a.va && QG_IN(a.ra * pitch + c0 + 3, n, 24)) ld4<T>(sa + c0, x);
            if (a.vb && QG_IN(a.rb * pitch + c0 + 3, n, 24)) ld4<T>(sb + c0, y);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) stp<T>(cb, c0 + shift + q, Cplx<T>{x[q], y[q]}, g.buf);
    }
    if (t == 0) stp<T>(cb, 0, Cplx<T>{T(0), T(0)}, g.buf);
}

// Between the two y transforms of phase 1: the mode-space solve, Eq. ialpha
// (OPY 1) or Eqs. isub-1/2 (OPY 2), written back as the next input.
template <typename T, int OPY, int RAD>
__device__ __forceinline__ void mode_solve(const SolveParams<T>& P, const PairAt& a,
                                           const Geo32& g, CT<T>* cb, int t,
                                           const T* __restrict__ lamy) {
    const T lxa = QG_IN(a.ra, P.mx + 1, 25) ? __ldg(P.lamx + a.ra) : T(1);
    const T lxb = QG_IN(a.rb, P.mx + 1, 25) ? __ldg(P.lamx + a.rb) : T(1);
#pragma unroll 4
    for (int i = 0; i < RAD / 2; ++i) {
        const int l = t + i * g.G;
        const Cplx<T> z = ldp<T>(cb, l, g.buf);
        const T Fa = T(-0.5) * z.y, Fb = T(0.5) * z.x;
        T x = T(0), y = T(0);
        if (l > 0 && a.va && QG_IN(l, P.my + 1, 26)) {
            const T ly = lamy[l];
            if (OPY == 1) {
                x = Fa * (P.scale / (lxa + ly));
                if (a.vb) y = Fb * (P.scale / (lxb + ly));
            } else {
                const T q1 = P.scale * Fa, q2 = P.scale * Fb;
                const T al = P.Ro * (lxa + ly);
                const T den = al * (al - P.f1 - P.f2);
                x = (al * q1 - P.f2 * q1 - P.f1 * q2) / den;
                y = (al * q2 - P.f2 * q1 - P.f1 * q2) / den;
            }
        }
        stp<T>(cb, l, Cplx<T>{x, y}, g.buf);
    }
}

// Write the transformed pair: F(a)_k = -Im Z_k / 2, F(b)_k = Re Z_k / 2.
//   phase 0: tr[k][ra - 1], tr[k][rb - 1] (k >= 1);
//   phase 1: work[j][ka - 1], work[j][kb - 1] (j >= 1);
//   phase 2: out[ra][k], out[rb][k], k = 0..N-1 (k = 0 is the wall).
template <typename T, int OPY, int RAD>
__device__ __forceinline__ void store_pair(const SolveParams<T>& P, int ph, const PairAt& a,
                                           const Geo32& g, const CT<T>* cb, int t) {
    if (!a.va) return;
#pragma unroll 4
    for (int i = 0; i < RAD / 2; ++i) {
        const int k = t + i * g.G;
        if (!QG_IN(px(k), g.buf, 27)) continue;
        const CT<T> z = cb[px(k)];
        const T fa = T(-0.5) * z.y, fb = T(0.5) * z.x;
        const long long nw = (long long)(P.my + 1) * P.ld;     // out, work
        const long long nt = (long long)(P.mx + 1) * P.ld_tr;  // tr
        if (ph == 2) {
            if (QG_IN((long long)a.ra * P.ld + k, nw, 28))
                P.out[a.layer][(size_t)a.ra * P.ld + k] = k == 0 ? T(0) : fa;
            if (a.vb && QG_IN((long long)a.rb * P.ld + k, nw, 28))
                P.out[a.layer][(size_t)a.rb * P.ld + k] = k == 0 ? T(0) : fb;
            continue;
        }
        if (k == 0) continue;
        if (ph == 0) {
            if (!QG_IN((long long)k * P.ld_tr + a.ra, nt, 29)) continue;
            T* d = P.tr[a.layer] + (size_t)k * P.ld_tr + (a.ra - 1);
            if (a.vb) st2<T>(d, fa, fb);
            else d[0] = fa;
        } else if (!QG_IN((long long)k * P.ld + a.rb - 1, nw, 30)) {
            continue;
        } else if (OPY == 2) {
            P.work[0][(size_t)k * P.ld + a.ra - 1] = fa;
            P.work[1][(size_t)k * P.ld + a.rb - 1] = fb;
        } else if (a.vb) {
            st2<T>(P.work[0] + (size_t)k * P.ld + a.ra - 1, fa, fb);
        } else {
            P.work[0][(size_t)k * P.ld + a.ra - 1] = fa;
        }
    }
}

// Shared-memory layout (bytes): pair buffers | x twiddles | y twiddles | lamy;
// the tables are staged only when they fit (Tabs::staged).
struct Tabs {
    int buf, tx, ty, ly, end;      // offsets and total
    int nx, ny, nl;                // bytes of each table
    bool staged;
};
__host__ __device__ inline int al16i(int v) { return (v + 15) / 16 * 16; }
__host__ __device__ inline Tabs tabs_for(int lgx, int lgy, int rad, int threads, int esz,
                                         int ntx, int nty, int my) {
    Tabs b;
    const int a1 = buf_cplx(lgx, rad, threads), a2 = buf_cplx(lgy, rad, threads);
    b.buf = al16i((a1 > a2 ? a1 : a2) * 2 * esz);
    b.nx = ntx * 2 * esz;
    b.ny = nty * 2 * esz;
    b.nl = ((my + 1 + 3) / 4 * 4) * esz;
    b.tx = b.buf;
    b.ty = b.tx + al16i(b.nx);
    b.ly = b.ty + al16i(b.ny);
    const int total = b.ly + al16i(b.nl);
    b.staged = total - b.buf <= 48 * 1024;
    b.end = b.staged ? total : b.buf;
    return b;
}

// Set the error flag of the solve, or of every member of a batch.
template <typename T, bool BATCH>
__device__ __forceinline__ void raise_err(const SolveParams<T>& P) {
    if constexpr (BATCH) {
        for (int i = 0; i < P.nbatch; ++i) atomicExch(P.batch[i].err, 1);
    } else {
        atomicExch(P.err, 1);
    }
}

// Phase 0 of a CTA whose two groups hold the pairs of rows r .. r + 3 of
// one layer: tr[k][r - 1 .. r + 2] for both pairs at once, one 16-byte
// store per k (the per-pair stores write 8 bytes of each 32-byte sector).
// r0, r1: the two groups' result buffers, final and visible to the CTA.
template <typename T>
__device__ __forceinline__ void store_quad(const SolveParams<T>& P, const PairAt& a0,
                                           const Geo32& g, const CT<T>* r0, const CT<T>* r1) {
    const long long nt = (long long)(P.mx + 1) * P.ld_tr;
    for (int k = threadIdx.x; k < g.N; k += blockDim.x) {
        if (k == 0 || !QG_IN(px(k), g.buf, 27)) continue;
        const CT<T> z0 = r0[px(k)], z1 = r1[px(k)];
        if (!QG_IN((long long)k * P.ld_tr + a0.ra + 2, nt, 29)) continue;
        T* d = P.tr[a0.layer] + (size_t)k * P.ld_tr + (a0.ra - 1);
        st4<T>(d, T(-0.5) * z0.y, T(0.5) * z0.x, T(-0.5) * z1.y, T(0.5) * z1.x);
    }
}

// One slot of phase ph: the pair of this thread's group, loaded, transformed
// (phase 1: forward, mode solve, inverse) and stored.
template <typename T, int OPY, int RAD>
__device__ __forceinline__ void solve_slot(const SolveParams<T>& P, int ph, int slot, int npairs,
                                           int per, int grp, int t, const Geo32& g, CT<T>* cb,
                                           CT<T>* cb2, const CT<T>* tw, const T* lamy,
                                           const Sync& sy) {
    const PairAt a = pair_at<T, OPY>(P, ph, slot * per + grp, npairs);
    load_pair<T, OPY, RAD>(P, ph, a, g, cb, t);
    const int nfft = ph == 1 ? 2 : 1;
    CT<T>* res = cb;
#pragma unroll 1
    for (int f = 0; f < nfft; ++f) {
        if (f == 1) mode_solve<T, OPY, RAD>(P, a, g, res, t, lamy);
        res = fft_rt<T, RAD>(res, res == cb ? cb2 : cb, t, g, tw, sy);
    }
    if (ph == 0 && per == 2) {
        // the same test in every thread of the CTA (it depends on the slot)
        const PairAt a0 = pair_at<T, OPY>(P, 0, slot * 2, npairs);
        const PairAt a1 = pair_at<T, OPY>(P, 0, slot * 2 + 1, npairs);
        if (a0.va && a0.vb && a1.va && a1.vb && a1.layer == a0.layer && a1.ra == a0.ra + 2 &&
            ((a0.ra - 1) & 3) == 0) {
            // group 1's buffers follow group 0's, and both results sit at
            // the same place in their group's pair of buffers
            const CT<T>* r0 = res - (size_t)grp * 2 * g.buf;
            __syncthreads();
            store_quad<T>(P, a0, g, r0, r0 + 2 * g.buf);
            __syncthreads();
            return;
        }
    }
    store_pair<T, OPY, RAD>(P, ph, a, g, res, t);
    sy.sync();
}

template <typename T, int OPY, int RAD>
__global__ void __launch_bounds__(max_cta(RAD, (int)sizeof(T)),
                                  (RAD == 8 && sizeof(T) == 4) ? 2 : 1)
solve32_kernel(SolveParams<T> P, int lgx, int lgy, Tabs tb) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    CT<T>* bufs = reinterpret_cast<CT<T>*>(smem);
    const CT<T>* ptx = P.ptx;
    const CT<T>* pty = P.pty;
    const T* lamy = P.lamy;
    const uint32_t bar = smem_u32(&mbar);
    if (tb.staged) {
        // the constant tables of both directions, copied once per CTA
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                         "r"(tb.nx + tb.ny + tb.nl) : "memory");
            if (tb.nx) bulk_copy(smem_u32(smem + tb.tx), P.ptx, tb.nx, bar);
            if (tb.ny) bulk_copy(smem_u32(smem + tb.ty), P.pty, tb.ny, bar);
            bulk_copy(smem_u32(smem + tb.ly), P.lamy, tb.nl, bar);
        }
        ptx = reinterpret_cast<const CT<T>*>(smem + tb.tx);
        pty = reinterpret_cast<const CT<T>*>(smem + tb.ty);
        lamy = reinterpret_cast<const T*>(smem + tb.ly);
    }
    // While the stage before is still writing them, touch (L2 prefetch) the
    // rows of the right-hand side this thread reads first, so that their
    // address translations are in place when the data is ready.
    if (!P.split || P.phase == 0) {
        const Geo32 g = geo32(lgx, RAD);
        const int npairs = (P.my / 2) * P.layers;
        const int per = blockDim.x / g.G;
        const PairAt a = pair_at<T, OPY>(P, 0, blockIdx.x * per + threadIdx.x / g.G, npairs);
        const int c0 = 4 * (threadIdx.x % g.G);
        if (a.va) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(P.in[a.layer][0] + (size_t)a.ra * P.ld + c0));
            if (a.vb)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(P.in[a.layer][0] + (size_t)a.rb * P.ld + c0));
        }
    }
    pdl_wait();
    pdl_trigger();   // the next fine stage may start staging its own inputs
    if (tb.staged) {
        const bool ok = mbar_wait(bar, 0, kSpin);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) raise_err<T, false>(P);
            (void)mbar_wait(bar, 0, kSpin);     // let copies in flight land
            return;
        }
    }
    const int ph0 = P.split ? P.phase : 0, ph1 = P.split ? P.phase + 1 : 3;
    unsigned g0 = 0;
    for (int ph = ph0; ph < ph1; ++ph) {
        if (ph > ph0 && !grid_sync(P.bar, P.bar_extra, kSpin, g0)) {
            if (threadIdx.x == 0) raise_err<T, false>(P);
            return;
        }
        if (ph + 1 < ph1) g0 = grid_gen(P.bar);
        const Geo32 g = geo32(ph == 1 ? lgy : lgx, RAD);
        const CT<T>* tw = ph == 1 ? pty : ptx;
        const int grp = threadIdx.x / g.G, t = threadIdx.x % g.G;
        CT<T>* cb = bufs + 2 * grp * g.buf;
        CT<T>* cb2 = cb + g.buf;
        const Sync sy{1 + grp, g.G};
        int npairs;
        if (ph == 1) npairs = OPY == 2 ? P.mx - 1 : P.mx / 2;
        else npairs = (P.my / 2) * P.layers;
        const int per = blockDim.x / g.G;
        const int nslots = (npairs + per - 1) / per;
        for (int slot = blockIdx.x; slot < nslots; slot += gridDim.x)
            solve_slot<T, OPY, RAD>(P, ph, slot, npairs, per, grp, t, g, cb, cb2, tw, lamy, sy);
    }
}

// Batched solve of an ensemble group as a work queue, without grid barriers
// (so that groups can run side by side on concurrent graph branches: a
// cooperative grid is not guaranteed to be co-resident with other work).
// The work items are the slots of the three phases of every member, phase
// by phase and member by member; CTAs claim them in that order from the
// counter q[0].  An item of phase ph >= 1 of member m first waits (bounded)
// until the q[2 + 3 m + ph - 1] items of phase ph - 1 of member m are done;
// those were claimed before it by CTAs that are running, and depend on no
// later item, so the wait ends without any co-residency.  A wait that runs
// out sets the member's error flag and the item is counted done unprocessed
// (its results are garbage, as the flag says).  The last CTA to leave resets
// the counters for the next launch.
__device__ __forceinline__ bool wait_count(const unsigned* c, unsigned want, int limit) {
    for (int i = 0; i < limit; ++i) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
        if (v >= want) return true;
    }
    return false;
}

template <typename T, int OPY, int RAD>
__device__ __forceinline__ void solve_queue(const SolveParams<T>& P, int lgx, int lgy,
                                            CT<T>* bufs, const CT<T>* ptx, const CT<T>* pty,
                                            const T* lamy, bool broken) {
    __shared__ int s_item;
    unsigned* q = P.bar;
    const int nb = P.nbatch;
    const Geo32 gx = geo32(lgx, RAD), gy = geo32(lgy, RAD);
    const int perx = blockDim.x / gx.G, pery = blockDim.x / gy.G;
    const int npx = P.my / 2, npy = P.mx / 2;            // one layer
    const int ns0 = (npx + perx - 1) / perx, ns1 = (npy + pery - 1) / pery;
    const int n0 = nb * ns0, n1 = n0 + nb * ns1, total = n1 + nb * ns0;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(q, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= total) break;
        int ph, m, slot;
        if (item < n0) {
            ph = 0; m = item / ns0; slot = item - m * ns0;
        } else if (item < n1) {
            ph = 1; m = (item - n0) / ns1; slot = item - n0 - m * ns1;
        } else {
            ph = 2; m = (item - n1) / ns0; slot = item - n1 - m * ns0;
        }
        const SolveMember<T>& M = P.batch[m];
        int ok = broken ? 0 : 1;
        if (ok && ph > 0 && threadIdx.x == 0)
            ok = wait_count(q + 2 + 3 * m + ph - 1, (unsigned)(ph == 1 ? ns0 : ns1), kSpin);
        if (__syncthreads_and(ok)) {
            const Geo32& g = ph == 1 ? gy : gx;
            const int grp = threadIdx.x / g.G, t = threadIdx.x % g.G;
            CT<T>* cb = bufs + 2 * grp * g.buf;
            CT<T>* cb2 = cb + g.buf;
            const Sync sy{1 + grp, g.G};
            SolveParams<T> Q = P;
#pragma unroll
            for (int k = 0; k < 4; ++k) Q.in[0][k] = M.in[k];
            Q.nin = M.nin;
            Q.part_px = M.part_px;
            Q.part_py = M.part_py;
            Q.tr[0] = M.tr;
            Q.work[0] = M.work;
            Q.out[0] = M.out;
            solve_slot<T, OPY, RAD>(Q, ph, slot, ph == 1 ? npy : npx, ph == 1 ? pery : perx, grp,
                                    t, g, cb, cb2, ph == 1 ? pty : ptx, lamy, sy);
            __syncthreads();
        } else if (threadIdx.x == 0) {
            atomicExch(M.err, 1);
        }
        if (threadIdx.x == 0) {
            // this CTA's stores of the item are ordered before the count by
            // the CTA barrier above and the release
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(q + 2 + 3 * m + ph)
                         : "memory");
        }
    }
    if (threadIdx.x == 0) {
        unsigned old;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(q + 1)
                     : "memory");
        if (old == gridDim.x - 1) {
            for (int i = 0; i < 2 + 3 * nb; ++i) q[i] = 0u;
        }
    }
}

template <typename T, int OPY, int RAD>
__global__ void __launch_bounds__(max_cta(RAD, (int)sizeof(T)),
                                  (RAD == 8 && sizeof(T) == 4) ? 2 : 1)
solve32_batch_kernel(SolveParams<T> P, int lgx, int lgy, Tabs tb) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    CT<T>* bufs = reinterpret_cast<CT<T>*>(smem);
    const CT<T>* ptx = P.ptx;
    const CT<T>* pty = P.pty;
    const T* lamy = P.lamy;
    const uint32_t bar = smem_u32(&mbar);
    if (tb.staged) {
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                         "r"(tb.nx + tb.ny + tb.nl) : "memory");
            if (tb.nx) bulk_copy(smem_u32(smem + tb.tx), P.ptx, tb.nx, bar);
            if (tb.ny) bulk_copy(smem_u32(smem + tb.ty), P.pty, tb.ny, bar);
            bulk_copy(smem_u32(smem + tb.ly), P.lamy, tb.nl, bar);
        }
        ptx = reinterpret_cast<const CT<T>*>(smem + tb.tx);
        pty = reinterpret_cast<const CT<T>*>(smem + tb.ty);
        lamy = reinterpret_cast<const T*>(smem + tb.ly);
    }
    pdl_wait();
    pdl_trigger();
    bool broken = false;
    if (tb.staged) {
        const bool ok = mbar_wait(bar, 0, kSpin);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) raise_err<T, true>(P);
            (void)mbar_wait(bar, 0, kSpin);     // let copies in flight land
            broken = true;   // claim items and count them done unprocessed
        }
    }
    solve_queue<T, OPY, RAD>(P, lgx, lgy, bufs, ptx, pty, lamy, broken);
}

int least_threads() {
    static int v = 0;
    if (!v) {
        v = 128;
        if (const char* e = std::getenv("QG_SOLVE32_THREADS")) {
            const int t = std::atoi(e);
            if (t >= 32 && t <= 256 && (t & (t - 1)) == 0) v = t;
        }
    }
    return v;
}

int log2i(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

template <typename T, int OPY, int RAD, bool BATCH = false>
cudaError_t launch32(const SolveParams<T>& P, cudaStream_t s) {
    void (*k)(SolveParams<T>, int, int, Tabs);
    if constexpr (BATCH) k = solve32_batch_kernel<T, OPY, RAD>;
    else k = solve32_kernel<T, OPY, RAD>;
    const int lgx = log2i(2 * P.mx), lgy = log2i(2 * P.my);
    const int threads = cta_threads(lgx, lgy, RAD, least_threads());
    const Tabs tb = tabs_for(lgx, lgy, RAD, threads, (int)sizeof(T),
                             (int)pass_table_size(2 * P.mx, RAD),
                             (int)pass_table_size(2 * P.my, RAD), P.my);
    const size_t sm = tb.end;
    int nsm = 0, per = 0;
    cudaError_t e = launch_shape(reinterpret_cast<const void*>(k), threads, sm, &per, &nsm);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    auto slots = [threads](int lg, int npairs) {
        const int pairs = threads / ((1 << lg) / RAD);
        return (npairs + pairs - 1) / pairs;
    };
    const int rows = (P.my / 2) * P.layers;
    const int cols = OPY == 2 ? P.mx - 1 : P.mx / 2;
    int want = slots(lgx, rows);
    if (slots(lgy, cols) > want) want = slots(lgy, cols);
    if (BATCH) want = P.nbatch * (2 * slots(lgx, rows) + slots(lgy, cols));   // queue items
    int grid = per * nsm;
    if (want < grid) grid = want;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    if (BATCH) {
        // the work queue needs no co-residency: a plain launch, allowed to
        // start while the kernel before it finishes (the table copies
        // precede the programmatic wait) unless no_pdl
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = P.no_pdl ? nullptr : at;
        cfg.numAttrs = P.no_pdl ? 0 : 1;
        return cudaLaunchKernelEx(&cfg, k, P, lgx, lgy, tb);
    }
    if (!P.split) {
        // cooperative (grid barriers), and allowed to start while the fine
        // stage before it finishes: the table copies precede the kernel's
        // programmatic wait, every read of the stage's output follows it
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 2;
        return cudaLaunchKernelEx(&cfg, k, P, lgx, lgy, tb);
    }
    SolveParams<T> Q = P;
    for (int ph = 0; ph < 3; ++ph) {
        Q.phase = ph;
        if ((e = cudaLaunchKernelEx(&cfg, k, Q, lgx, lgy, tb)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

// lengths 2N = 2^lg with G = 2^lg / RAD threads per pair within one CTA
// (G <= max_cta(RAD, esz))
bool solve32_supports(int mx, int my, int rad, size_t esz) {
    const int lx = log2i(2 * mx), ly = log2i(2 * my), lr = log2i(rad);
    const int lt = log2i(max_cta(rad, (int)esz));
    return (rad == 8 || rad == 16 || rad == 32) && is_pow2(mx) && is_pow2(my) && lx >= lr &&
           ly >= lr && lx <= lr + lt && ly <= lr + lt;
}

size_t solve32_smem_bytes(int mx, int my, size_t esz, int rad) {
    const int lx = log2i(2 * mx), ly = log2i(2 * my);
    const int th = cta_threads(lx, ly, rad, least_threads());
    return tabs_for(lx, ly, rad, th, (int)esz, (int)pass_table_size(2 * mx, rad),
                    (int)pass_table_size(2 * my, rad), my).end;
}

template <typename T>
cudaError_t launch_solve32(const SolveParams<T>& P, int rad, cudaStream_t s) {
    if (!solve32_supports(P.mx, P.my, rad, sizeof(T)) || !P.ptx || !P.pty)
        return cudaErrorInvalidValue;
    if (P.batch) {
        if (P.layers != 1 || P.split || P.nbatch < 1) return cudaErrorInvalidValue;
        if (rad == 8) return launch32<T, 1, 8, true>(P, s);
        if (rad == 16) return launch32<T, 1, 16, true>(P, s);
        return launch32<T, 1, 32, true>(P, s);
    }
    if (rad == 8)
        return P.layers == 2 ? launch32<T, 2, 8>(P, s) : launch32<T, 1, 8>(P, s);
    if (rad == 16)
        return P.layers == 2 ? launch32<T, 2, 16>(P, s) : launch32<T, 1, 16>(P, s);
    return P.layers == 2 ? launch32<T, 2, 32>(P, s) : launch32<T, 1, 32>(P, s);
}

QG_BOUNDS_QUERY(bounds_site_solve32)

template cudaError_t launch_solve32<float>(const SolveParams<float>&, int, cudaStream_t);
template cudaError_t launch_solve32<double>(const SolveParams<double>&, int, cudaStream_t);

}  // namespace qg
