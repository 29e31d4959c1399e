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
// t = 0..2N-1, stored in the working precision and staged in shared memory
// when it is small.  A CTA holds `lanes` complex sequences of length 2N in
// shared memory (stride 4N + 2 reals); each is worked on by TPR = 2N/(4 NB)
// threads doing NB radix-4 butterflies per pass.  Every pass reads its
// operands into registers, synchronises and writes in place.
//
// The 2-D solve is three launches of one kernel:
//   x pass   rows of the elliptic-grid field (the restriction arrives as the
//            sum of up to four partial planes) -> x-spectrum written
//            transposed, so the y pass reads contiguous rows;
//   y pass   rows of the transposed array: forward DST over y, division by
//            the eigenvalues of Eq. ialpha (or the 2x2 system of Eqs.
//            isub-1/2 for two layers, the two layers of a mode forming one
//            sequence pair), inverse DST, written back untransposed;
//   x pass   inverse transform of the rows -> streamfunction.
// All reads are contiguous; only the stores are strided.
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
template <typename T, int NB, typename TW>
__device__ __forceinline__ void fft_pass4(T* buf, const Geo& g, int Ns, const TW* tw) {
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

template <typename T, int NB, typename TW>
__device__ __forceinline__ void fft_inplace(T* buf, const Geo& g, const TW* tw) {
    int Ns = 1;
    if (g.logL & 1) {
        fft_pass2_first<T, NB>(buf, g);
        Ns = 2;
    }
    for (; Ns < g.L; Ns <<= 2) fft_pass4<T, NB>(buf, g, Ns, tw);
}

// z_j = (a_j, b_j) and its odd extension z_{2N-j} = -z_j (j >= 1); j = 0
// also clears z_N.
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

// Byte offsets of the shared-memory regions of one dst_pass CTA.
__host__ __device__ constexpr size_t al16(size_t v) { return (v + 15) / 16 * 16; }
__host__ __device__ inline size_t lamy_offset(int N, int lanes, size_t esz) {
    return al16((size_t)lanes * lane_stride(N) * esz);
}
__host__ __device__ inline size_t tw_offset(int N, int lanes, size_t esz, bool lamy) {
    return al16(lamy_offset(N, lanes, esz) + (lamy ? (size_t)N * esz : 0));
}

// One DST pass over sequence pairs; see DstPass in qg_internal.cuh.
template <typename T, int NB, int OP>
__global__ void __launch_bounds__(512)
dst_pass_kernel(DstPass<T> d) {
    using C = typename Cx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geo g = make_geo(d.N, NB);
    const int lanes = blockDim.x / g.TPR;
    const int N = d.N;
    T* base = reinterpret_cast<T*>(smem_raw);
    T* buf = base + g.lane * lane_stride(N);
    // constant tables (twiddles, lamy) go to shared memory by bulk copies
    // issued before waiting on the previous kernel
    __shared__ __align__(8) uint64_t mbar;
    const uint32_t bar = smem_u32(&mbar);
    T* slamy = reinterpret_cast<T*>(smem_raw + lamy_offset(N, lanes, sizeof(T)));
    C* stw = reinterpret_cast<C*>(smem_raw + tw_offset(N, lanes, sizeof(T), OP != 0));
    const bool staged = (OP != 0) || d.tw_in_smem;
    if (staged) {
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint32_t tb = d.tw_in_smem ? (uint32_t)(2 * N * sizeof(C)) : 0u;
            const uint32_t lb = OP != 0 ? (uint32_t)(N * sizeof(T)) : 0u;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         ::"r"(bar), "r"(tb + lb) : "memory");
            if (tb) bulk_copy(smem_u32(stw), d.tw, tb, bar);
            if (lb) bulk_copy(smem_u32(slamy), d.lamy, lb, bar);
        }
    }
    const C* tw = d.tw_in_smem ? stw : d.tw;
    pdl_wait();

    // sequence pair of this lane: rows ra / rb of planes pa / pb
    const int pair = blockIdx.x * lanes + g.lane;
    int ra, rb, pa, pb;
    if (d.pair_planes) {
        ra = rb = 1 + pair;
        pa = 0;
        pb = 1;
    } else {
        ra = 1 + 2 * pair;
        rb = ra + 1;
        pa = pb = 0;
    }
    const bool va = ra <= d.nrows, vb = rb <= d.nrows;
    // all input loads first (2 NB elements of each sequence per thread)
    constexpr int JPT = 2 * NB;
    T av[JPT], bv[JPT];
    const bool rpa = d.nin > 1 && (ra % d.part_py) == 0;
    const bool rpb = d.nin > 1 && (rb % d.part_py) == 0;
    const size_t oa = (size_t)ra * d.ld_in, ob = (size_t)rb * d.ld_in;
#pragma unroll
    for (int it = 0; it < JPT; ++it) {
        const int j = g.t + it * g.TPR;
        T a = T(0), b = T(0);
        if (j > 0) {
            if (va) a = __ldg(d.in[pa][0] + oa + j);
            if (vb) b = __ldg(d.in[pb][0] + ob + j);
            if (d.nin > 1) {
                const bool cx = (j % d.part_px) == 0;
                if (va) {
                    if (cx) a += __ldg(d.in[pa][1] + oa + j);
                    if (rpa) a += __ldg(d.in[pa][2] + oa + j);
                    if (cx && rpa) a += __ldg(d.in[pa][3] + oa + j);
                }
                if (vb) {
                    if (cx) b += __ldg(d.in[pb][1] + ob + j);
                    if (rpb) b += __ldg(d.in[pb][2] + ob + j);
                    if (cx && rpb) b += __ldg(d.in[pb][3] + ob + j);
                }
            }
        }
        av[it] = a;
        bv[it] = b;
    }
#pragma unroll
    for (int it = 0; it < JPT; ++it) put_pair(buf, N, g.t + it * g.TPR, av[it], bv[it]);
    bool ok = true;
    if (staged) ok = mbar_wait(bar, 0, 1 << 22);
    __syncthreads();
    if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0 && d.err) atomicExch(d.err, 1);
        return;
    }
    fft_inplace<T, NB>(buf, g, tw);

    if (OP != 0) {
        // mode space: F_l(a) = -Im Z_l / 2, F_l(b) = Re Z_l / 2
        for (int l = g.t; l < N; l += g.TPR) {
            T a = T(0), b = T(0);
            if (l > 0) {
                const T Fa = T(-0.5) * buf[2 * l + 1];
                const T Fb = T(0.5) * buf[2 * l];
                const T ly = slamy[l];
                if (OP == 1) {
                    // one layer: psihat = scale Qhat / (lamx[k] + lamy[l])
                    if (va) a = Fa * (d.scale / (d.lamx[ra] + ly));
                    if (vb) b = Fb * (d.scale / (d.lamx[rb] + ly));
                } else if (va) {
                    // two layers, Eqs. isub-1/2 with alpha = Ro (lamx + lamy)
                    const T q1 = d.scale * Fa, q2 = d.scale * Fb;
                    const T al = d.Ro * (d.lamx[ra] + ly);
                    const T den = al * (al - d.f1 - d.f2);
                    a = (al * q1 - d.f2 * q1 - d.f1 * q2) / den;
                    b = (al * q2 - d.f2 * q1 - d.f1 * q2) / den;
                }
            }
            put_pair(buf, N, l, a, b);
        }
        __syncthreads();
        fft_inplace<T, NB>(buf, g, tw);
    }
    pdl_trigger();

    // outputs: F_k(a) -> (plane pa, row ra), F_k(b) -> (plane pb, row rb)
    if (!d.transpose_out) {
        T* oa = d.out[pa] + (size_t)ra * d.ld_out;
        T* ob = d.out[pb] + (size_t)rb * d.ld_out;
        for (int k = g.t; k < N; k += g.TPR) {
            if (va) oa[k] = (k == 0) ? T(0) : T(-0.5) * buf[2 * k + 1];
            if (vb) ob[k] = (k == 0) ? T(0) : T(0.5) * buf[2 * k];
        }
    } else {
        // element k of row r goes to out[k][r]: consecutive threads take
        // consecutive rows of one k
        const int nseq = 2 * lanes;
        for (int idx = threadIdx.x; idx < (N - 1) * nseq; idx += blockDim.x) {
            const int c = idx % nseq, k = 1 + idx / nseq;
            const int ln = c >> 1, part = c & 1;
            const int pr = blockIdx.x * lanes + ln;
            int r, pl;
            if (d.pair_planes) {
                r = 1 + pr;
                pl = part;
            } else {
                r = 1 + 2 * pr + part;
                pl = 0;
            }
            if (r > d.nrows) continue;
            const T* bl = base + ln * lane_stride(N);
            d.out[pl][(size_t)k * d.ld_out + r] =
                part ? T(0.5) * bl[2 * k] : T(-0.5) * bl[2 * k + 1];
        }
    }
}

}  // namespace

// one radix-4 butterfly per thread and pass, up to 512 threads per pair
static int pick_nb(int N) {
    const int L = 2 * N;
    int nb = L / 2048;
    if (nb < 1) nb = 1;
    if (nb > 8) nb = 8;
    return nb;
}

static constexpr size_t kSmemCap = 200 * 1024;
static constexpr size_t kTwiddleSmemCap = 32 * 1024;

DstLaunch dst_config(int N, size_t esz, bool pair_planes) {
    (void)pair_planes;
    DstLaunch c;
    c.nb = pick_nb(N);
    const int tpr = (2 * N) / (4 * c.nb);
    int lanes = 1;

    c.lanes = lanes;
    return c;
}

size_t dst_max_smem() { return kSmemCap; }
size_t dst_lane_bytes(int N, size_t esz) { return esz * (size_t)lane_stride(N); }

template <typename K>
static cudaError_t allow_smem(K k) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
}

cudaError_t dst_prepare_kernels() {
    cudaError_t e = cudaSuccess;
#define QG_ALLOW(T, NB)                                                         \
    if (e == cudaSuccess) e = allow_smem(dst_pass_kernel<T, NB, 0>);          \
    if (e == cudaSuccess) e = allow_smem(dst_pass_kernel<T, NB, 1>);          \
    if (e == cudaSuccess) e = allow_smem(dst_pass_kernel<T, NB, 2>);
    QG_ALLOW(float, 1) QG_ALLOW(float, 2) QG_ALLOW(float, 4) QG_ALLOW(float, 8)
    QG_ALLOW(double, 1) QG_ALLOW(double, 2) QG_ALLOW(double, 4) QG_ALLOW(double, 8)
#undef QG_ALLOW
    return e;
}

template <typename T, int NB, int OP>
static cudaError_t launch_nb(const DstPass<T>& d, dim3 grid, dim3 block, size_t sm,
                             cudaStream_t s, bool pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, dst_pass_kernel<T, NB, OP>, d);
}

template <typename T>
cudaError_t launch_dst_pass(DstPass<T> d, int op, DstLaunch cfg, cudaStream_t s, bool pdl) {
    using C = typename Cx<T>::type;
    const int tpr = (2 * d.N) / (4 * cfg.nb);
    const dim3 block(tpr * cfg.lanes);
    const int pairs = d.pair_planes ? d.nrows : (d.nrows + 1) / 2;
    const dim3 grid((pairs + cfg.lanes - 1) / cfg.lanes);
    // smem: sequence buffers, lamy (op != 0), twiddles (16-byte aligned)
    const size_t twb = sizeof(C) * 2 * (size_t)d.N;
    d.tw_in_smem = twb <= kTwiddleSmemCap ? 1 : 0;
    const size_t sm = tw_offset(d.N, cfg.lanes, sizeof(T), op != 0) + (d.tw_in_smem ? twb : 0);
    if (d.nin > 1 && (d.part_px <= 0 || d.part_py <= 0)) return cudaErrorInvalidValue;
    cudaError_t e = cudaErrorInvalidValue;
#define QG_CASE(NB)                                                                  \
    case NB:                                                                         \
        e = op == 0 ? launch_nb<T, NB, 0>(d, grid, block, sm, s, pdl)               \
          : op == 1 ? launch_nb<T, NB, 1>(d, grid, block, sm, s, pdl)               \
                    : launch_nb<T, NB, 2>(d, grid, block, sm, s, pdl);              \
        break;
    switch (cfg.nb) {
        QG_CASE(1) QG_CASE(2) QG_CASE(4) QG_CASE(8)
        default: break;
    }
#undef QG_CASE
    return e;
}

template cudaError_t launch_dst_pass<float>(DstPass<float>, int, DstLaunch, cudaStream_t, bool);
template cudaError_t launch_dst_pass<double>(DstPass<double>, int, DstLaunch, cudaStream_t, bool);

}  // namespace qg
