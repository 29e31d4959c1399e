// Elliptic solve of Section 4.3 for long sequences (engine 50).
//
// The same transforms as the warp-group engine of solve32.cu: the x pass of
// the right-hand side, the y pass with the mode-space solve of Eq. ialpha
// (or Eqs. isub-1/2 for two layers), and the inverse x pass, each a DST-I
// of two real sequences computed as one complex FFT of length L = 2N of
// their odd extensions (F(a)_k = -Im Z_k / 2, F(b)_k = Re Z_k / 2).  The
// engine is laid out for grids whose passes stream through HBM (the full
// 2048 x 4096 grid, l = 0):
//
//   * G = L/16 threads per sequence pair, three plain launches (one per
//     pass) chained by programmatic dependent launch, so there is no grid
//     barrier and each pass takes the CTA size and register budget of its
//     own length; an ensemble group's batch runs instead as one launch, a
//     work queue over the items of the three passes of every member
//     (stream_queue_kernel);
//   * thread t holds the 16 values x[t + G r] in registers.  The first
//     radix-16 pass works on the values the thread loaded from global
//     memory, and the last pass leaves X[t + G s] in registers (a Stockham
//     pass of sub-transform size L/16 writes its output in natural order),
//     so an FFT of length L = 16^p 2^q takes p + (q > 0) - 1 shared-memory
//     exchanges (L = 4096: two; 8192: three) between the global load and
//     the global store;
//   * the odd extension is completed in shared memory: each thread stores
//     its z[t + G r], r < 8, and reads back the reflected -z[L - m];
//   * the y pass keeps the forward spectrum in registers for the mode-space
//     solve and starts the inverse transform from there;
//   * one shared buffer of L complex per pair: every pass reads all its
//     operands into registers before any thread of the pair writes;
//   * the passes that write transposed (x forward into tr, y into work) hold
//     2 or 4 pairs per CTA, each on its own named barrier, and stage their
//     outputs in shared memory so that each row receives 2 PPC consecutive
//     values (FP32, 4 pairs: a whole 32-byte sector) instead of one 8-byte
//     pair per row and thread;
//   * the length is a template parameter: every shared-memory, twiddle and
//     global offset of a pass is a constant from a per-thread base.
//
// Twiddles come from the radix-16 pass tables of the warp-group engine
// (pass_table(L, 16), FP64-generated): a radix-16 pass loads w, w^2, w^4
// and w^8 and forms the other powers, the remainder pass one power per
// radix and multiplies by 16th roots of unity.
#include <cuda_runtime.h>

#include "bounds.cuh"
#include "dst_engine.cuh"
#include "qg_internal.cuh"

namespace qg {
namespace {

using namespace eng;

// padded slot of complex element m (one pad per 16 spreads the strided
// stores of the passes over the banks)
__host__ __device__ constexpr int sp(int m) { return m + (m >> 4); }
__host__ __device__ constexpr int buf_elems(int L) { return sp(L) + 2; }

// Shared-memory access at padded slot i (a slot, not an element index).
template <typename T>
__device__ __forceinline__ Cplx<T> ldsl(const CT<T>* b, int i, int lim) {
    (void)lim;
    if (!QG_IN(i, lim, 61)) return Cplx<T>{T(0), T(0)};
    const CT<T> v = b[i];
    return Cplx<T>{v.x, v.y};
}
template <typename T>
__device__ __forceinline__ void stsl(CT<T>* b, int i, Cplx<T> v, int lim) {
    (void)lim;
    if (!QG_IN(i, lim, 62)) return;
    CT<T> w;
    w.x = v.x;
    w.y = v.y;
    b[i] = w;
}

// FFT length L = 2^LG = 16^NP 2^REM, G = L/16 threads per pair (LG >= 8, so
// G is a multiple of 16 and sp(a + r G) = sp(a) + r sp(G) for a < G).
template <int LG>
struct Len {
    static constexpr int L = 1 << LG, N = L / 2, G = L / 16, NP = LG / 4, REM = LG % 4;
    static constexpr int LIM = buf_elems(L);
    static constexpr int SG = G + G / 16;   // sp(G)
};

// Barrier of the G threads of one pair (named barrier 1 + group), or of the
// whole CTA when it holds one pair.
struct GSync {
    int id, n;
    bool cta;
    __device__ __forceinline__ void sync() const {
        if (cta) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
    }
};

// Offset of pass p's block in pass_table(L, 16): blocks of 16 x 16^q for
// q = 1 .. p - 1.
__host__ __device__ constexpr int tw_off(int p) {
    int o = 0, ns = 16;
    for (int q = 1; q < p; ++q, ns *= 16) o += 16 * ns;
    return o;
}

// Store the outputs of radix-16 pass q (sub-transform size NS = 16^q) to
// (t - k) 16 + k + r NS, k = t mod NS, in padded slots.
template <typename T, int LG, int NS>
__device__ __forceinline__ void put_pass(const Cplx<T> (&v)[16], CT<T>* buf, int t) {
    using Ln = Len<LG>;
    int base;
    if constexpr (NS == 1) {
        base = 17 * t;                      // sp(16 t + r) = 17 t + r
    } else {
        const int k = t & (NS - 1);
        const int d = (t - k) * 16 + k;
        base = d + (d >> 4);                // sp(d + r NS) = sp(d) + r sp(NS)
    }
    constexpr int step = NS == 1 ? 1 : NS + NS / 16;
#pragma unroll
    for (int r = 0; r < 16; ++r) stsl<T>(buf, base + r * step, v[out_slot<16>(r)], Ln::LIM);
}

// Radix-16 pass p >= 1 (sub-transform size 16^p): read t + r G, twiddle,
// 16-point DFT.
template <typename T, int LG, int P>
__device__ __forceinline__ void mid_pass(Cplx<T> (&v)[16], CT<T>* buf, int t,
                                         const CT<T>* __restrict__ tw, const GSync& sy) {
    using Ln = Len<LG>;
    constexpr int NS = 1 << (4 * P);
    put_pass<T, LG, NS / 16>(v, buf, t);
    sy.sync();
    const int rb = t + (t >> 4);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = ldsl<T>(buf, rb + r * Ln::SG, Ln::LIM);
    sy.sync();
    // twiddles w^r = e^{-2 pi i r k / (16 NS)}: w, w^2, w^4 and w^8 from the
    // table, the other powers as products (at most three roundings deep)
    const CT<T>* tp = tw + tw_off(P) + (t & (NS - 1));
    Cplx<T> w[16];
    {
        const CT<T> a = __ldg(tp + NS), b = __ldg(tp + 2 * NS), c = __ldg(tp + 4 * NS),
                    d = __ldg(tp + 8 * NS);
        w[1] = Cplx<T>{a.x, a.y};
        w[2] = Cplx<T>{b.x, b.y};
        w[4] = Cplx<T>{c.x, c.y};
        w[8] = Cplx<T>{d.x, d.y};
    }
    w[3] = cmul(w[2], w[1].x, w[1].y);
    w[5] = cmul(w[4], w[1].x, w[1].y);
    w[6] = cmul(w[4], w[2].x, w[2].y);
    w[7] = cmul(w[4], w[3].x, w[3].y);
#pragma unroll
    for (int r = 1; r < 8; ++r) w[8 + r] = cmul(w[8], w[r].x, w[r].y);
#pragma unroll
    for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], w[r].x, w[r].y);
    dft<T, 16>(v);
}

// e^{-2 pi i m / 16}, m = 0..15, as compile-time constants
template <typename T>
__device__ __forceinline__ Cplx<T> w16(int m) {
    const T c1 = K16<T>::c1, s1 = K16<T>::s1, r2 = K16<T>::r2;
    const T cs[4] = {T(1), c1, r2, s1}, sn[4] = {T(0), s1, r2, c1};
    const int q = m >> 2, e = m & 3;
    const T c = cs[e], s = sn[e];   // e^{-i pi e / 8} = c - i s
    switch (q) {                    // times (-i)^q
        case 0: return Cplx<T>{c, -s};
        case 1: return Cplx<T>{-s, -c};
        case 2: return Cplx<T>{-c, s};
        default: return Cplx<T>{s, c};
    }
}

// The remainder pass (radix R = 2^REM, B = 16/R butterflies j = t + b G per
// thread, sub-transform size L/R): output X[t + G (b + B r)] to v[b + B r].
template <typename T, int LG, int R>
__device__ __forceinline__ void rem_pass(Cplx<T> (&v)[16], CT<T>* buf, int t,
                                         const CT<T>* __restrict__ tw, const GSync& sy) {
    using Ln = Len<LG>;
    constexpr int B = 16 / R, NSR = Ln::L / R, SNSR = NSR + NSR / 16;
    put_pass<T, LG, (1 << (4 * Ln::NP)) / 16>(v, buf, t);
    sy.sync();
    const int rb = t + (t >> 4);
    Cplx<T> u[B][R];
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) u[b][r] = ldsl<T>(buf, rb + b * Ln::SG + r * SNSR, Ln::LIM);
    sy.sync();
    // twiddle of butterfly j = t + b G: e^{-2 pi i r j / L} = e^{-2 pi i r t / L}
    // e^{-2 pi i r b / 16} (G = L / 16): R - 1 table loads per thread
    const CT<T>* tp = tw + tw_off(Ln::NP) + t;
    Cplx<T> wt[R];
#pragma unroll
    for (int r = 1; r < R; ++r) {
        const CT<T> a = __ldg(tp + r * NSR);
        wt[r] = Cplx<T>{a.x, a.y};
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
            const Cplx<T> c = w16<T>((r * b) & 15);
            const Cplx<T> w = b == 0 ? wt[r] : cmul(wt[r], c.x, c.y);
            u[b][r] = cmul(u[b][r], w.x, w.y);
        }
        dft<T, R>(u[b]);
#pragma unroll
        for (int r = 0; r < R; ++r) v[b + B * r] = u[b][out_slot<R>(r)];
    }
}

// Forward FFT of length L: on entry v[r] = x[t + G r], on return
// v[s] = X[t + G s].  buf is free on entry and on return.
template <typename T, int LG>
__device__ __forceinline__ void fft16s(Cplx<T> (&v)[16], CT<T>* buf, int t,
                                       const CT<T>* __restrict__ tw, const GSync& sy) {
    using Ln = Len<LG>;
    dft<T, 16>(v);   // pass 0: sub-transform size 1, no twiddles
    if constexpr (Ln::NP >= 2) mid_pass<T, LG, 1>(v, buf, t, tw, sy);
    if constexpr (Ln::NP >= 3) mid_pass<T, LG, 2>(v, buf, t, tw, sy);
    if constexpr (Ln::REM == 0) {
        // the last radix-16 pass had sub-transform size G: X[t + G r] is in
        // slot out_slot(r)
        Cplx<T> o[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) o[r] = v[out_slot<16>(r)];
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = o[r];
    } else {
        rem_pass<T, LG, (1 << Ln::REM)>(v, buf, t, tw, sy);
    }
}

// Odd extension: v[r] = z[t + G r] holds for r < 8 on entry (z_0 = 0); the
// values r >= 8 are -z[c G - t] for c = 16 - r (0 at c G - t = N), read from
// the other threads' values through buf.
template <typename T, int LG>
__device__ __forceinline__ void reflect(Cplx<T> (&v)[16], CT<T>* buf, int t, const GSync& sy) {
    using Ln = Len<LG>;
    const int rb = t + (t >> 4);
#pragma unroll
    for (int r = 0; r < 8; ++r) stsl<T>(buf, rb + r * Ln::SG, v[r], Ln::LIM);
    if (t == 0) stsl<T>(buf, sp(Ln::N), Cplx<T>{T(0), T(0)}, Ln::LIM);
    sy.sync();
    // sp(c G - t) = c sp(G) - (t + ceil(t / 16))
    const int u = t + ((t + 15) >> 4);
#pragma unroll
    for (int r = 8; r < 16; ++r) {
        const Cplx<T> z = ldsl<T>(buf, (16 - r) * Ln::SG - u, Ln::LIM);
        v[r] = Cplx<T>{-z.x, -z.y};
    }
    sy.sync();
}

// Rows a (and b when vb) of the right-hand side, elements j = t + G r,
// r < 8 (j = 0 is the wall: 0): plane 0, plus plane 2 on rows with
// row % part_py == 0, plus planes 1 and 3 at columns j % part_px == 0
// (periods are powers of two: masks).
// Every load of a row is issued before any sum.
template <typename T, int G>
__device__ __forceinline__ void load_rhs(const SolveParams<T>& P, const T* const (&in)[4], int ra,
                                         int rb, bool va, bool vb, int t, Cplx<T> (&v)[16]) {
    const long long n = (long long)(P.my + 1) * P.ld;
    const size_t oa = (size_t)ra * P.ld + t, ob = (size_t)rb * P.ld + t;
    const T* pa = in[0] + (va ? oa : 0);
    const T* pb = in[0] + (vb ? ob : 0);
    T a[8], b[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const bool j0 = r == 0 && t == 0;
        const bool ia = va && !j0 && QG_IN(oa + r * G, n, 63);
        const bool ib = vb && !j0 && QG_IN(ob + r * G, n, 63);
        a[r] = ia ? __ldg(pa + r * G) : T(0);
        b[r] = ib ? __ldg(pb + r * G) : T(0);
    }
    if (P.nin > 1) {
        const bool ya = (ra & (P.part_py - 1)) == 0, yb = (rb & (P.part_py - 1)) == 0;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int j = t + r * G;
            const bool j0 = j == 0;
            const bool ia = va && !j0 && QG_IN(oa + r * G, n, 63);
            const bool ib = vb && !j0 && QG_IN(ob + r * G, n, 63);
            const bool cx = (j & (P.part_px - 1)) == 0;
            if (ia && ya) a[r] += __ldg(in[2] + oa + r * G);
            if (ib && yb) b[r] += __ldg(in[2] + ob + r * G);
            if (ia && cx) {
                a[r] += __ldg(in[1] + oa + r * G);
                if (ya) a[r] += __ldg(in[3] + oa + r * G);
            }
            if (ib && cx) {
                b[r] += __ldg(in[1] + ob + r * G);
                if (yb) b[r] += __ldg(in[3] + ob + r * G);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = Cplx<T>{a[r], b[r]};
}

// Rows a and b of a scratch array (element j at column j - 1, j = 0: 0),
// from row offsets oa, ob of arrays sa, sb with n elements.
template <typename T, int G>
__device__ __forceinline__ void load_rows(const T* sa, const T* sb, bool va, bool vb,
                                          long long oa, long long ob, long long n, int t,
                                          Cplx<T> (&v)[16]) {
    const T* pa = sa + (va ? oa + t - 1 : 0);
    const T* pb = sb + (vb ? ob + t - 1 : 0);
    T a[8], b[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const bool j0 = r == 0 && t == 0;
        const bool ia = va && !j0 && QG_IN(oa + t - 1 + r * G, n, 64);
        const bool ib = vb && !j0 && QG_IN(ob + t - 1 + r * G, n, 64);
        a[r] = ia ? __ldg(pa + r * G) : T(0);
        b[r] = ib ? __ldg(pb + r * G) : T(0);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = Cplx<T>{a[r], b[r]};
}

// Pairs per CTA of the passes that write transposed: `want`, fewer while
// the CTA would exceed 1024 threads (FP32) or 512 (FP64, 128 registers per
// thread) or 140 KB of shared memory.
constexpr int kPpcX = 4, kPpcY = 4;   // x forward pass, y pass
template <typename T>
__host__ __device__ constexpr int ppc_for(int lg, int want) {
    int p = want;
    while (p > 1 && (((1 << lg) / 16) * p > (sizeof(T) == 4 ? 1024 : 512) ||
                     (long long)p * buf_elems(1 << lg) * (long long)sizeof(T) * 2 > 140 * 1024))
        p /= 2;
    return p;
}
// Threads per CTA and the register budget: 64 per thread at 512 threads
// and more, 80 below (FP32); 128 (FP64).
template <typename T>
__host__ __device__ constexpr int minb_for(int threads) {
    const int regs = sizeof(T) == 8 ? 128 : (threads >= 512 ? 64 : 80);
    const int b = 65536 / (threads * regs);
    return b < 1 ? 1 : (b > 16 ? 16 : b);
}

// Staging pitch (in T) of the transposed outputs of PPC pairs: 2 PPC
// values per spectral index, padded against bank conflicts.
__host__ __device__ constexpr int stage_pitch(int ppc) { return 2 * ppc + (ppc >= 4 ? 4 : 2); }

// One pass of the solve for PPC sequence pairs per CTA (pair
// blockIdx.x PPC + group, one group of G threads each).
//   YP false, PH 0: rows ra, rb of the right-hand side -> tr[k][ra - 1, rb - 1];
//   YP false, PH 2: rows ra, rb of work (element j at column j - 1) -> out;
//   YP true:        x-modes ka, kb: rows of tr (element j at column j - 1),
//                   forward transform, mode-space solve, inverse transform
//                   -> work[l][ka - 1, kb - 1] (OPY 2: layers 0 and 1 of
//                   x-mode ka).
// The transposed outputs (tr, work) of the CTA's pairs are staged in shared
// memory and written as runs of 2 PPC values per row.
// One work item: PPC sequence pairs (pair blk PPC + group, one group of G
// threads each) of phase PH, with P's arrays (a member's, for batches).
// Every thread of the CTA takes part.
template <typename T, int OPY, int PH, int LG, int PPC>
__device__ __forceinline__ void stream_item(const SolveParams<T>& P, int npairs, int blk,
                                            unsigned char* smem) {
    using Ln = Len<LG>;
    constexpr bool YP = PH == 1;
    constexpr int G = Ln::G;
    const int grp = PPC == 1 ? 0 : (int)threadIdx.x / G;
    const int t = (int)threadIdx.x - grp * G;
    const int pair0 = blk * PPC, pair = pair0 + grp;
    const bool vp = pair < npairs;
    CT<T>* buf = reinterpret_cast<CT<T>*>(smem) + grp * Ln::LIM;
    const GSync sy{1 + grp, G, PPC == 1};
    int layer = 0, ra, rb;
    bool vb;
    if (YP) {
        if (OPY == 2) {
            ra = rb = 1 + pair;
            vb = vp;
        } else {
            ra = 1 + 2 * pair;
            rb = ra + 1;
            vb = vp && rb <= P.mx - 1;
        }
    } else {
        const int ppl = P.my / 2;
        layer = pair0 / ppl;       // ppl is a multiple of PPC: one layer per CTA
        ra = 1 + 2 * (pair - layer * ppl);
        rb = ra + 1;
        vb = vp && rb <= P.my - 1;
    }
    const CT<T>* tw = YP ? P.pty : P.ptx;
    // the layer's arrays, selected without indexing (an indexed parameter
    // array would be copied to local memory)
    const bool l1 = layer != 0;
    const T* const in[4] = {l1 ? P.in[1][0] : P.in[0][0], l1 ? P.in[1][1] : P.in[0][1],
                            l1 ? P.in[1][2] : P.in[0][2], l1 ? P.in[1][3] : P.in[0][3]};
    T* const trl = l1 ? P.tr[1] : P.tr[0];
    T* const workl = l1 ? P.work[1] : P.work[0];
    T* const outl = l1 ? P.out[1] : P.out[0];

    Cplx<T> v[16];
    if (YP) {
        const long long n = (long long)(P.mx + 1) * P.ld_tr;
        load_rows<T, G>(P.tr[0], P.tr[OPY == 2 ? 1 : 0], vp, vb, (long long)ra * P.ld_tr,
                        (long long)rb * P.ld_tr, n, t, v);
    } else if (PH == 0) {
        load_rhs<T, G>(P, in, ra, rb, vp, vb, t, v);
    } else {
        const long long n = (long long)(P.my + 1) * P.ld;
        load_rows<T, G>(workl, workl, vp, vb, (long long)ra * P.ld,
                        (long long)rb * P.ld, n, t, v);
    }
    reflect<T, LG>(v, buf, t, sy);
    fft16s<T, LG>(v, buf, t, tw, sy);

    if (YP) {
        // mode-space solve of the modes l = t + G s, s < 8 (l = 0: the wall)
        const T lxa = QG_IN(ra, P.mx + 1, 66) ? __ldg(P.lamx + ra) : T(1);
        const T lxb = QG_IN(rb, P.mx + 1, 66) ? __ldg(P.lamx + rb) : T(1);
        const T* ly_t = P.lamy + t;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const T Fa = T(-0.5) * v[s].y, Fb = T(0.5) * v[s].x;
            T x = T(0), y = T(0);
            if (vp && (s > 0 || t > 0) && QG_IN(t + s * G, P.my + 1, 67)) {
                const T ly = __ldg(ly_t + s * G);
                if (OPY == 1) {
                    x = Fa * (P.scale / (lxa + ly));
                    if (vb) y = Fb * (P.scale / (lxb + ly));
                } else {
                    const T q1 = P.scale * Fa, q2 = P.scale * Fb;
                    const T al = P.Ro * (lxa + ly);
                    const T den = al * (al - P.f1 - P.f2);
                    x = (al * q1 - P.f2 * q1 - P.f1 * q2) / den;
                    y = (al * q2 - P.f2 * q1 - P.f1 * q2) / den;
                }
            }
            v[s] = Cplx<T>{x, y};
        }
        reflect<T, LG>(v, buf, t, sy);
        fft16s<T, LG>(v, buf, t, tw, sy);
    }

    // F(a)_k = -Im Z_k / 2, F(b)_k = Re Z_k / 2 for k = t + G s < N
    if constexpr (PH == 2) {
        const long long nw = (long long)(P.my + 1) * P.ld;
        T* oa = outl + (size_t)ra * P.ld + t;
        T* ob = outl + (size_t)rb * P.ld + t;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const T fa = T(-0.5) * v[s].y, fb = T(0.5) * v[s].x;
            const bool k0 = s == 0 && t == 0;
            if (vp && QG_IN((long long)ra * P.ld + t + s * G, nw, 70)) oa[s * G] = k0 ? T(0) : fa;
            if (vb && QG_IN((long long)rb * P.ld + t + s * G, nw, 70)) ob[s * G] = k0 ? T(0) : fb;
        }
    } else {
        // transposed outputs: stage [k][2 group + (0: a, 1: b)], then write runs
        constexpr int SP = stage_pitch(PPC), W = 2 * PPC;
        T* stg = reinterpret_cast<T*>(smem);
        __syncthreads();   // every group is done with its FFT buffer
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            CT<T> o;
            o.x = T(-0.5) * v[s].y;
            o.y = T(0.5) * v[s].x;
            const int i = (t + s * G) * SP + 2 * grp;
            if (QG_IN(i + 1, (long long)PPC * Ln::LIM * 2, 71))
                *reinterpret_cast<CT<T>*>(stg + i) = o;
        }
        __syncthreads();
        // thread e of the CTA writes column q = e mod W of rows
        // k = e / W + i G / 2 (G PPC threads cover G / 2 rows per step)
        const int q = (int)threadIdx.x % W, k0 = (int)threadIdx.x / W;
        constexpr int KSTEP = G / 2, ITER = Ln::N / KSTEP;
        if (YP) {
            // work[l][c], l = 1..my-1; OPY 1: c = 2 pair0 + q; OPY 2: layer
            // q % 2 at column pair0 + q / 2
            const long long nw = (long long)(P.my + 1) * P.ld;
            const int c = OPY == 1 ? 2 * pair0 + q : pair0 + (q >> 1);
            T* dst = (OPY == 1 || !(q & 1) ? P.work[0] : P.work[1]) + c;
            const bool vc = c <= P.mx - 2;
#pragma unroll 4
            for (int i = 0; i < ITER; ++i) {
                const int k = k0 + i * KSTEP;
                if (k > 0 && vc && QG_IN((long long)k * P.ld + c, nw, 72))
                    dst[(size_t)k * P.ld] = stg[k * SP + q];
            }
        } else {
            // tr[k][c], k = 1..mx-1, c = 2 (pair0 - layer ppl) + q
            const long long ntr = (long long)(P.mx + 1) * P.ld_tr;
            const int c = 2 * (pair0 - layer * (P.my / 2)) + q;
            T* dst = trl + c;
            const bool vc = c <= P.my - 2;
#pragma unroll 4
            for (int i = 0; i < ITER; ++i) {
                const int k = k0 + i * KSTEP;
                if (k > 0 && vc && QG_IN((long long)k * P.ld_tr + c, ntr, 69))
                    dst[(size_t)k * P.ld_tr] = stg[k * SP + q];
            }
        }
    }
}

// One launch per pass.  Batches (ensembles, one layer): member
// blockIdx.x / cpm takes CTAs blockIdx.x mod cpm, with its arrays from
// P.batch.
template <typename T, int OPY, int PH, int LG, int PPC>
__global__ void __launch_bounds__(Len<LG>::G * PPC, minb_for<T>(Len<LG>::G * PPC))
stream_kernel(SolveParams<T> Pin, int npairs, int cpm) {
    extern __shared__ __align__(16) unsigned char smem[];
    SolveParams<T> P = Pin;
    int blk = blockIdx.x;
    if (Pin.batch) {
        const int m = blk / cpm;
        blk -= m * cpm;
        const SolveMember<T>& M = Pin.batch[m];
#pragma unroll
        for (int q = 0; q < 4; ++q) P.in[0][q] = M.in[q];
        P.nin = M.nin;
        P.part_px = M.part_px;
        P.part_py = M.part_py;
        P.tr[0] = M.tr;
        P.work[0] = M.work;
        P.out[0] = M.out;
    }
    pdl_wait();
    pdl_trigger();
    stream_item<T, OPY, PH, LG, PPC>(P, npairs, blk, smem);
}

// Batched solve of an ensemble group in one launch (one layer, y length
// twice the x length): a work queue over the items of the three passes of
// every member, claimed in order from the counter q[0] (pass by pass,
// member by member).  An item of pass ph >= 1 of member m first waits
// (bounded) until the q[2 + 3 m + ph - 1] items of the pass before are
// done; those were claimed earlier by CTAs that are running and depend on
// no later item, so the wait ends without any co-residency.  A wait that
// runs out sets the member's error flag and the item is counted done
// unprocessed.  The last CTA to leave resets the counters for the next
// launch.  The CTA has BT threads: BT / G_x pairs per x item, BT / G_y per
// y item.
constexpr int kQueueSpin = 1 << 22;

__device__ __forceinline__ bool wait_done(const unsigned* c, unsigned want, int limit) {
    for (int i = 0; i < limit; ++i) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
        if (v >= want) return true;
    }
    return false;
}

template <typename T, int LGX, int BT>
__global__ void __launch_bounds__(BT, minb_for<T>(BT))
stream_queue_kernel(SolveParams<T> P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    constexpr int LGY = LGX + 1;
    constexpr int PX = BT / Len<LGX>::G, PY = BT / Len<LGY>::G;
    unsigned* q = P.bar;
    const int nb = P.nbatch;
    const int rows = P.my / 2, cols = P.mx / 2;
    const int n0i = (rows + PX - 1) / PX, n1i = (cols + PY - 1) / PY;
    const int e0 = nb * n0i, e1 = e0 + nb * n1i, total = e1 + nb * n0i;
    pdl_wait();
    pdl_trigger();
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(q, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= total) break;
        int ph, m, blk;
        if (item < e0) {
            ph = 0; m = item / n0i; blk = item - m * n0i;
        } else if (item < e1) {
            ph = 1; m = (item - e0) / n1i; blk = item - e0 - m * n1i;
        } else {
            ph = 2; m = (item - e1) / n0i; blk = item - e1 - m * n0i;
        }
        const SolveMember<T>& M = P.batch[m];
        int ok = 1;
        if (ph > 0 && threadIdx.x == 0)
            ok = wait_done(q + 2 + 3 * m + ph - 1, (unsigned)(ph == 1 ? n0i : n1i), kQueueSpin);
        if (__syncthreads_and(ok)) {
            SolveParams<T> Q = P;
#pragma unroll
            for (int k = 0; k < 4; ++k) Q.in[0][k] = M.in[k];
            Q.nin = M.nin;
            Q.part_px = M.part_px;
            Q.part_py = M.part_py;
            Q.tr[0] = M.tr;
            Q.work[0] = M.work;
            Q.out[0] = M.out;
            if (ph == 0) stream_item<T, 1, 0, LGX, PX>(Q, rows, blk, smem);
            else if (ph == 1) stream_item<T, 1, 1, LGY, PY>(Q, cols, blk, smem);
            else stream_item<T, 1, 2, LGX, PX>(Q, rows, blk, smem);
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

// Lengths 2^LG of the engine: L = 512 .. 16384 (FP32), .. 8192 (FP64).
constexpr int kMinLg = 9, kMaxLg = 14;

template <typename T, int OPY, int PH, int LG>
cudaError_t launch_pass(const SolveParams<T>& P, int npairs, cudaStream_t s) {
    constexpr int PPC = PH == 2 ? 1 : ppc_for<T>(LG, PH == 0 ? kPpcX : kPpcY);
    constexpr int G = Len<LG>::G;
    const int cpm = (npairs + PPC - 1) / PPC;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cpm * (P.batch ? P.nbatch : 1));
    cfg.blockDim = dim3(G * PPC);
    const size_t fft_bytes = (size_t)PPC * Len<LG>::LIM * sizeof(CT<T>);
    const size_t stg_bytes = PH == 2 ? 0 : (size_t)Len<LG>::N * stage_pitch(PPC) * sizeof(T);
    cfg.dynamicSmemBytes = fft_bytes > stg_bytes ? fft_bytes : stg_bytes;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    // (ensemble branches run side by side: a dependent started early would
    // hold SM resources idle, so their launches may go without)
    cfg.attrs = P.no_pdl ? nullptr : at;
    cfg.numAttrs = P.no_pdl ? 0 : 1;
    auto k = stream_kernel<T, OPY, PH, LG, PPC>;
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cfg.dynamicSmemBytes);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, k, P, npairs, cpm);
}

template <typename T, int OPY, int PH>
cudaError_t launch_lg(const SolveParams<T>& P, int lg, int npairs, cudaStream_t s) {
    switch (lg) {
        case 9: return launch_pass<T, OPY, PH, 9>(P, npairs, s);
        case 10: return launch_pass<T, OPY, PH, 10>(P, npairs, s);
        case 11: return launch_pass<T, OPY, PH, 11>(P, npairs, s);
        case 12: return launch_pass<T, OPY, PH, 12>(P, npairs, s);
        case 13: return launch_pass<T, OPY, PH, 13>(P, npairs, s);
        case 14:
            if constexpr (sizeof(T) == 4) return launch_pass<T, OPY, PH, 14>(P, npairs, s);
            return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int OPY>
cudaError_t launch_all(const SolveParams<T>& P, cudaStream_t s) {
    const int lgx = ilog2(2 * P.mx), lgy = ilog2(2 * P.my);
    const int rows = (P.my / 2) * P.layers;
    const int cols = OPY == 2 ? P.mx - 1 : P.mx / 2;
    cudaError_t e = launch_lg<T, OPY, 0>(P, lgx, rows, s);
    if (e == cudaSuccess) e = launch_lg<T, OPY, 1>(P, lgy, cols, s);
    if (e == cudaSuccess) e = launch_lg<T, OPY, 2>(P, lgx, rows, s);
    return e;
}

// The work-queue launch of a batch: the CTA size and pairs per item.
template <typename T>
constexpr int queue_threads(int lgx) {
    const int gy = (1 << (lgx + 1)) / 16;
    const int maxt = sizeof(T) == 4 ? 1024 : 512;
    return 4 * gy < maxt ? 4 * gy : maxt;
}

template <typename T, int LGX>
cudaError_t launch_queue_lg(const SolveParams<T>& P, cudaStream_t s) {
    constexpr int BT = queue_threads<T>(LGX);
    constexpr int PX = BT / Len<LGX>::G, PY = BT / Len<LGX + 1>::G;
    auto k = stream_queue_kernel<T, LGX, BT>;
    size_t sm = (size_t)PX * Len<LGX>::LIM * sizeof(CT<T>);
    const size_t smy = (size_t)PY * Len<LGX + 1>::LIM * sizeof(CT<T>);
    const size_t stx = (size_t)Len<LGX>::N * stage_pitch(PX) * sizeof(T);
    const size_t sty = (size_t)Len<LGX + 1>::N * stage_pitch(PY) * sizeof(T);
    for (size_t v : {smy, stx, sty}) sm = v > sm ? v : sm;
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, BT, sm)) != cudaSuccess)
        return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    const int rows = P.my / 2, cols = P.mx / 2;
    const int total = P.nbatch * (2 * ((rows + PX - 1) / PX) + (cols + PY - 1) / PY);
    int grid = per * nsm;
    if (total < grid) grid = total;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(BT);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = P.no_pdl ? nullptr : at;
    cfg.numAttrs = P.no_pdl ? 0 : 1;
    return cudaLaunchKernelEx(&cfg, k, P);
}

}  // namespace

// Batches of one-layer grids with my = 2 mx and 2 mx = 2^9 .. 2^11 run as
// one work-queue launch; other batches as three launches.
bool stream_queue_ok(int mx, int my, int layers) {
    if (layers != 1 || my != 2 * mx || !is_pow2(mx)) return false;
    const int lx = ilog2(2 * mx);
    return lx >= 9 && lx <= 11;
}

bool stream_supports(int mx, int my, size_t esz) {
    if (!is_pow2(mx) || !is_pow2(my)) return false;
    const int lx = ilog2(2 * mx), ly = ilog2(2 * my);
    const int hi = esz == 4 ? kMaxLg : kMaxLg - 1;
    return lx >= kMinLg && ly >= kMinLg && lx <= hi && ly <= hi;
}

template <typename T>
cudaError_t launch_solve_stream(const SolveParams<T>& P, cudaStream_t s) {
    if (!stream_supports(P.mx, P.my, sizeof(T)) || !P.ptx || !P.pty ||
        (P.batch && (P.layers != 1 || P.nbatch < 1)))
        return cudaErrorInvalidValue;
    if (P.batch && stream_queue_ok(P.mx, P.my, P.layers) && P.bar) {
        switch (ilog2(2 * P.mx)) {
            case 9: return launch_queue_lg<T, 9>(P, s);
            case 10: return launch_queue_lg<T, 10>(P, s);
            default: return launch_queue_lg<T, 11>(P, s);
        }
    }
    return P.layers == 2 ? launch_all<T, 2>(P, s) : launch_all<T, 1>(P, s);
}

QG_BOUNDS_QUERY(bounds_site_stream)

template cudaError_t launch_solve_stream<float>(const SolveParams<float>&, cudaStream_t);
template cudaError_t launch_solve_stream<double>(const SolveParams<double>&, cudaStream_t);

}  // namespace qg
