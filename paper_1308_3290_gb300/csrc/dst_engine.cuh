// Device-side DST-I engine of the elliptic solver (solve.cu).
//
// The paper's sine sums (Eqs. ifft-1/2, ffft-1/2) are unnormalised type-I
// discrete sine transforms, F_k = sum_{j=1}^{N-1} f_j sin(pi j k / N), for a
// power-of-two N.  The engine transforms two real sequences a, b at once:
//
//   z_j = a_j + i b_j (j = 1..N-1),  z_0 = z_N = 0,  z_{2N-j} = -z_j,
//   Z = FFT_{2N}(z),
//   F_k(a) = -Im Z_k / 2,   F_k(b) = Re Z_k / 2,   k = 1..N-1.
//
// The odd extension of a real sequence has a purely imaginary DFT equal to
// -2i times its DST-I, so packing b as the imaginary part puts its transform
// in the real part.  Every output is a plain FFT output: there is no
// recurrence, so the FP32 rounding error grows like log N (a half-length
// transform whose odd outputs come from a running sum, tried first, lost
// accuracy like sqrt N and missed the FP32 tolerance at N >= 1024).
//
// The FFT is a Stockham autosort transform in shared memory with base
// radix E = 16 (radix-16 passes, then one radix-2, 4 or 8 pass for the
// remaining factor of L = 2N) or E = 4 (radix-4 passes and one radix-2
// pass): a pass with sub-transform size Ns reads element j + r L/R,
// multiplies it by e^{-2 pi i r k/(R Ns)} (k = j mod Ns) and writes the
// R-point DFT to (j - k) R + k + r Ns.  Each thread does nb base-radix
// butterflies per pass with its operands in registers, so a pass is one
// read phase and one write phase around a block barrier.  E = 16 needs
// fewer passes and instructions, E = 4 four times as many threads per
// sequence pair; which is faster depends on how many pairs a grid offers,
// so the solver times both (see the autotuner in api.cu).  Complex element m
// of a sequence lives at m + m/16 (one pad per 16) to spread the strided
// writes over the banks.  Twiddles come from one FP64-generated table per N,
// tw[t] = e^{i pi t/N}, t = 0..2N-1, in the working precision.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qg_internal.cuh"

namespace qg {
namespace eng {

template <typename T>
using CT = typename Cx<T>::type;

template <typename T>
struct Cplx {
    T x, y;
};

__host__ __device__ __forceinline__ int pidx(int m) { return m + (m >> 4); }
// complex elements of one padded sequence of length 2N (+ 2 spare)
__host__ __device__ constexpr int lane_cplx(int N) { return 2 * N + (N >> 3) + 2; }

template <typename T>
__device__ __forceinline__ Cplx<T> ldc(const CT<T>* b, int m) {
    const CT<T> v = b[pidx(m)];
    return Cplx<T>{v.x, v.y};
}
template <typename T>
__device__ __forceinline__ void stc(CT<T>* b, int m, Cplx<T> v) {
    CT<T> w;
    w.x = v.x;
    w.y = v.y;
    b[pidx(m)] = w;
}
template <typename T>
__device__ __forceinline__ Cplx<T> cadd(Cplx<T> a, Cplx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ Cplx<T> csub(Cplx<T> a, Cplx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ Cplx<T> cmi(Cplx<T> a) { return {a.y, -a.x}; }   // -i a
template <typename T>
__device__ __forceinline__ Cplx<T> cmul(Cplx<T> a, T wx, T wy) {
    return {a.x * wx - a.y * wy, a.x * wy + a.y * wx};
}
// a * conj(w)
template <typename T, typename W>
__device__ __forceinline__ Cplx<T> cmul_conj(Cplx<T> a, W w) {
    return {a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y};
}

// forward 4-point DFT in place
template <typename T>
__device__ __forceinline__ void dft4(Cplx<T>& a0, Cplx<T>& a1, Cplx<T>& a2, Cplx<T>& a3) {
    const Cplx<T> t0 = cadd(a0, a2), t1 = csub(a0, a2);
    const Cplx<T> t2 = cadd(a1, a3), t3 = cmi(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

// cos(pi/8), sin(pi/8), sqrt(1/2)
template <typename T> struct K16 {
    static constexpr T c1 = T(0.92387953251128675613);
    static constexpr T s1 = T(0.38268343236508977173);
    static constexpr T r2 = T(0.70710678118654752440);
};

// Forward R-point DFTs in place.  Radix 16 and 8 leave output r in slot
// (r mod 4) * (R/4) + r / 4; radix 4 and 2 in slot r (see out_slot).
template <typename T, int R>
__device__ __forceinline__ void dft(Cplx<T>* v) {
    if (R == 2) {
        const Cplx<T> a = v[0];
        v[0] = cadd(a, v[1]);
        v[1] = csub(a, v[1]);
    } else if (R == 4) {
        dft4(v[0], v[1], v[2], v[3]);
    } else if (R == 8) {
        // n = 2 n1 + n2, k = k1 + 4 k2
        dft4(v[0], v[2], v[4], v[6]);
        dft4(v[1], v[3], v[5], v[7]);
        // v[1 + 2 k1] *= e^{-2 pi i k1/8}
        v[3] = cmul(v[3], K16<T>::r2, -K16<T>::r2);
        v[5] = cmi(v[5]);
        v[7] = cmul(v[7], -K16<T>::r2, -K16<T>::r2);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            const Cplx<T> a = v[2 * k1];
            v[2 * k1] = cadd(a, v[2 * k1 + 1]);
            v[2 * k1 + 1] = csub(a, v[2 * k1 + 1]);
        }
    } else {   // R == 16: n = 4 n1 + n2, k = k1 + 4 k2
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) dft4(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
        // slot 4 k1 + n2 holds y[n2][k1]; multiply by e^{-2 pi i n2 k1/16}
        const T c1 = K16<T>::c1, s1 = K16<T>::s1, r2 = K16<T>::r2;
        v[5] = cmul(v[5], c1, -s1);      // n2 = 1, k1 = 1
        v[9] = cmul(v[9], r2, -r2);      //         k1 = 2
        v[13] = cmul(v[13], s1, -c1);    //         k1 = 3
        v[6] = cmul(v[6], r2, -r2);      // n2 = 2, k1 = 1
        v[10] = cmi(v[10]);              //         k1 = 2
        v[14] = cmul(v[14], -r2, -r2);   //         k1 = 3
        v[7] = cmul(v[7], s1, -c1);      // n2 = 3, k1 = 1
        v[11] = cmul(v[11], -r2, -r2);   //         k1 = 2
        v[15] = cmul(v[15], -c1, s1);    //         k1 = 3
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) dft4(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    }
}
template <int R>
__device__ __forceinline__ constexpr int out_slot(int r) {
    return R >= 8 ? (r & 3) * (R / 4) + (r >> 2) : r;
}

struct Geo {
    int nb;     // base-radix butterflies per thread and pass
    int N;      // DST length parameter (N - 1 unknowns)
    int L;      // complex FFT length, 2N
    int logL;
    int TPR;    // threads per sequence pair, L / (E nb)
    int t;      // thread index within the pair
    int lane;   // pair index within the CTA
};

template <int E>
__device__ __forceinline__ Geo make_geo(int N, int nb) {
    Geo g;
    g.nb = nb;
    g.N = N;
    g.L = 2 * N;
    g.logL = 31 - __clz(g.L);
    g.TPR = g.L / (E * nb);
    g.t = threadIdx.x % g.TPR;
    g.lane = threadIdx.x / g.TPR;
    return g;
}

// One Stockham pass of radix R (E / R butterflies per thread and unit nb).
template <typename T, int NBM, int E, int R>
__device__ __forceinline__ void fft_pass(CT<T>* cb, const Geo& g, int Ns, const CT<T>* tw) {
    constexpr int PER = E / R;
    const int stride = g.L / R;
    const int tstep = g.L / (R * Ns);
    Cplx<T> v[NBM * PER][R];
#pragma unroll
    for (int b = 0; b < NBM * PER; ++b) {
        if (b >= g.nb * PER) break;
        const int j = g.t + b * g.TPR;
        const int k = j & (Ns - 1);
#pragma unroll
        for (int r = 0; r < R; ++r) v[b][r] = ldc<T>(cb, j + r * stride);
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[b][r] = cmul_conj(v[b][r], tw[r * k * tstep]);
        }
        dft<T, R>(v[b]);
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < NBM * PER; ++b) {
        if (b >= g.nb * PER) break;
        const int j = g.t + b * g.TPR;
        const int k = j & (Ns - 1);
        const int d = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) stc<T>(cb, d + r * Ns, v[b][out_slot<R>(r)]);
    }
    __syncthreads();
}

// Forward complex FFT of length L in place.  Every thread of the CTA must
// call it (it contains block barriers).
template <typename T, int NBM, int E>
__device__ __forceinline__ void fft_inplace(CT<T>* cb, const Geo& g, const CT<T>* tw) {
    int Ns = 1;
    if (E == 16) {
        const int p16 = g.logL >> 2;
        for (int p = 0; p < p16; ++p, Ns <<= 4) fft_pass<T, NBM, 16, 16>(cb, g, Ns, tw);
        switch (g.logL & 3) {
            case 1: fft_pass<T, NBM, 16, 2>(cb, g, Ns, tw); break;
            case 2: fft_pass<T, NBM, 16, 4>(cb, g, Ns, tw); break;
            case 3: fft_pass<T, NBM, 16, 8>(cb, g, Ns, tw); break;
            default: break;
        }
    } else {
        const int p4 = g.logL >> 1;
        for (int p = 0; p < p4; ++p, Ns <<= 2) fft_pass<T, NBM, 4, 4>(cb, g, Ns, tw);
        if (g.logL & 1) fft_pass<T, NBM, 4, 2>(cb, g, Ns, tw);
    }
}

// z_j = (a_j, b_j) and its odd extension z_{2N-j} = -z_j (j >= 1); j = 0
// also clears z_N.
template <typename T>
__device__ __forceinline__ void put_pair(CT<T>* cb, int N, int j, T a, T b) {
    if (j == 0) {
        stc<T>(cb, 0, Cplx<T>{T(0), T(0)});
        stc<T>(cb, N, Cplx<T>{T(0), T(0)});
    } else {
        stc<T>(cb, j, Cplx<T>{a, b});
        stc<T>(cb, 2 * N - j, Cplx<T>{-a, -b});
    }
}
// F_k(a) and F_k(b) of a transformed pair
template <typename T>
__device__ __forceinline__ T dst_a(const CT<T>* cb, int k) { return T(-0.5) * cb[pidx(k)].y; }
template <typename T>
__device__ __forceinline__ T dst_b(const CT<T>* cb, int k) { return T(0.5) * cb[pidx(k)].x; }

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// 1-D bulk copies of the constant tables into shared memory on an mbarrier.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int limit) {
    for (int i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// Generation of the grid barrier `bar` (thread 0; 0 elsewhere).  Read in
// the phase before the barrier, off its critical path: the generation
// cannot advance before this CTA arrives.
__device__ __forceinline__ unsigned grid_gen(const unsigned* bar) {
    unsigned g = 0;
    if (threadIdx.x == 0)
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(bar + 1) : "memory");
    return g;
}

// Grid-wide barrier with a bounded wait.  bar[0] counts arrivals, bar[1] is
// the generation, g0 its value from grid_gen in this phase.  The arrival is
// an acq_rel atomic, so the CTA's writes of the phase (ordered before thread
// 0 by the CTA barrier) are visible to whoever acquires after it; the last of
// gridDim.x + extra arrivals resets the count and advances the generation
// with a release, and the others poll the generation with acquire loads.
// Returns false (on every thread) when the wait ran out.
__device__ inline bool grid_sync(unsigned* bar, unsigned extra, int limit, unsigned g0) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        unsigned old;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
                     : "=r"(old) : "l"(bar) : "memory");
        if (old == gridDim.x - 1 + extra) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(bar) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar + 1) : "memory");
        } else {
            for (int i = 0;; ++i) {
                unsigned g;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];"
                             : "=r"(g) : "l"(bar + 1) : "memory");
                if (g != g0) break;
                if (i >= limit) {
                    ok = 0;
                    break;
                }
            }
        }
    }
    return __syncthreads_and(ok) != 0;
}

}  // namespace eng
}  // namespace qg
