// Elliptic solve of Section 4.3 in matrix form on the tensor cores, for small
// elliptic grids.
//
// The sine sums of Eqs. ffft-1/2 and ifft-1/2 are products with the sine
// matrices S_x[i][k] = sin(pi i k / Mx) and S_y[j][l] = sin(pi j l / My)
// (interior indices from 1), both symmetric, so the solve of Eq. ialpha on
// the (My-1) x (Mx-1) right-hand side Q (rows y, columns x) is
//
//     Psi = S_y ((S_y Q S_x) o Inv) S_x,   Inv[l][k] = (2/Mx)(2/My) / lambda_kl,
//
// four dense products and one element-wise scaling.  One CTA of 16 warps
// does all of it: the sine matrices are copied into shared memory by 1-D
// bulk copies (before the programmatic wait: they are constants), the
// right-hand side (the sum of the restriction's partial planes) is read
// into shared memory, and each product writes its result to the other of
// two shared-memory work arrays; the scaling by Inv (an FP64-evaluated
// table) is the epilogue of the second product and the last product writes
// psi to global memory.
//
// Precision: the products run on the TF32 tensor path with FP32
// accumulation, each FP32 operand x split into two TF32 numbers hi = rn(x)
// and lo = rn(x - hi) and every product formed as lo*hi + hi*lo + hi*hi (the
// lo*lo term lies below FP32 rounding), which gives FP32 accuracy.  The
// tensor core's accumulation rounds toward zero: fed the running sum as its
// addend, it shrank every output by about 2^-23 per k-step, a bias that
// built up to 2e-6 relative over the four products (measured, 64 x 64).
// Each k-step therefore accumulates its three products from zero and the
// running sum is kept with ordinary round-to-nearest FP32 adds.
//
// The products are issued with the warp-level mma.sync (m16n8k8, TF32).
// The grids this engine serves are at most 128 nodes on a side, so a whole
// solve is a few million multiply-adds in a chain of four dependent
// products inside one CTA: its time is the latency of that chain, not the
// tensor throughput that tcgen05's 64- and 128-row tiles and TMEM
// accumulators are built for.
//
// Shared-memory pitches avoid bank conflicts in the fragment loads: an
// operand read as the A (row-major 16 x 8) fragment has a pitch of 4 mod 32
// floats (the eight rows of a fragment column start 4 banks apart), one read
// as the B (8 x 8) fragment a pitch of 8 or 24 mod 32 (its four rows start
// 8 banks apart).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "dst_engine.cuh"
#include "bounds.cuh"
#include "solve_mtx.h"

namespace qg {
namespace {

using namespace eng;

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kSpin = 1 << 22;

__host__ __device__ inline int r16(int v) { return (v + 15) / 16 * 16; }

// Layout of one elliptic grid, in floats.  m, n: interior columns (x) and
// rows (y); mp, np: padded to multiples of 16 (zeros beyond m, n).  S_x is
// mp x mp (pitch ldx, a B operand), S_y np x np (pitch ldy, an A operand);
// the work arrays U, V (and U2, V2 of the second layer) are np x mp with
// pitch lda (as an A operand) or ldb (as a B operand).  Shared memory:
// S_x | S_y | U | V | U2 | V2.  Global table: S_x | S_y | Inv (np x mp,
// pitch mp).
struct MtxGeo {
    int m, n, mp, np;
    int ldx, ldy, lda, ldb;
    int sx, sy, u, v, u2, v2, end;
    int tinv, tend;
};
__host__ __device__ inline MtxGeo mtx_geo(int mx, int my, int layers = 1) {
    MtxGeo g;
    g.m = mx - 1;
    g.n = my - 1;
    g.mp = r16(g.m);
    g.np = r16(g.n);
    g.ldx = g.mp + 8;
    g.ldy = g.np + 4;
    g.lda = g.mp + 4;
    g.ldb = g.mp + 8;
    g.sx = 0;
    g.sy = g.sx + g.mp * g.ldx;
    g.u = g.sy + g.np * g.ldy;
    g.v = g.u + g.np * g.ldb;
    g.u2 = g.v + g.np * g.ldb;
    g.v2 = g.u2 + g.np * g.ldb;
    g.end = layers == 2 ? g.v2 + g.np * g.ldb : g.u2;
    g.tinv = g.u;
    g.tend = g.tinv + g.np * g.mp;
    return g;
}

__device__ __forceinline__ uint32_t tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
// x = hi + lo to about 22 bits, both TF32
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = tf32_rn(x);
    lo = tf32_rn(x - __uint_as_float(hi));
}
// c += a b for one 16 x 8 x 8 TF32 tile
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C = A B for the np x mp result, A np x K (pitch lda), B K x mp (pitch
// ldb), K a multiple of 16.  A warp computes 16 x 16 tiles (two 16 x 8 mma
// columns sharing the A fragment); the fragment of lane (q = lane / 4,
// t = lane % 4) holds A rows q, q + 8 at columns t, t + 4 of the k-step, B
// rows t, t + 4 at column q, and C rows q, q + 8 at columns 2t, 2t + 1.
// epi(r, c, v0, v1) receives the outputs at (r, c) and (r, c + 1).
template <typename Epi>
__device__ __forceinline__ void mm3(const float* A, int lda, const float* B, int ldb, int K,
                                    const MtxGeo& g, Epi epi) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = lane >> 2, t = lane & 3;
    const int tc = g.mp / 16, nt = (g.np / 16) * tc;
    for (int tile = warp; tile < nt; tile += kWarps) {
        const int r0 = (tile / tc) * 16, c0 = (tile % tc) * 16;
        float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
        const float* a = A + (r0 + q) * lda + t;
        const float* b = B + t * ldb + c0 + q;
#pragma unroll 2
        for (int k0 = 0; k0 < K; k0 += 8) {
            uint32_t ah[4], al[4];
            split_tf32(a[k0], ah[0], al[0]);
            split_tf32(a[k0 + 8 * lda], ah[1], al[1]);
            split_tf32(a[k0 + 4], ah[2], al[2]);
            split_tf32(a[k0 + 8 * lda + 4], ah[3], al[3]);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                uint32_t bh0, bl0, bh1, bl1;
                split_tf32(b[k0 * ldb + 8 * j], bh0, bl0);
                split_tf32(b[(k0 + 4) * ldb + 8 * j], bh1, bl1);
                // the k-step's three products into a fresh accumulator,
                // small terms first, then one rounded FP32 add to the sum
                float p[4] = {0.f, 0.f, 0.f, 0.f};
                mma_tf32(p, al, bh0, bh1);
                mma_tf32(p, ah, bl0, bl1);
                mma_tf32(p, ah, bh0, bh1);
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[j][e] += p[e];
            }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int c = c0 + 8 * j + 2 * t;
            epi(r0 + q, c, acc[j][0], acc[j][1]);
            epi(r0 + q + 8, c, acc[j][2], acc[j][3]);
        }
    }
}

// The right-hand side of one layer (planes `in`) at interior node (x = c + 1,
// y = r + 1) into A (np x mp, pitch lda): the sum of the restriction's
// partial planes as in the FFT engines.
__device__ __forceinline__ void load_q(const SolveParams<float>& P, const float* const (&in)[4],
                                       float* A, const MtxGeo& g) {
    for (int i = threadIdx.x; i < g.np * g.mp; i += kThreads) {
        const int r = i / g.mp, c = i - r * g.mp;
        float v = 0.f;
        if (r < g.n && c < g.m &&
            QG_IN((long long)(r + 1) * P.ld + c + 1, (long long)(P.my + 1) * P.ld, 51)) {
            const int y = r + 1, x = c + 1;
            const size_t off = (size_t)y * P.ld + x;
            v = __ldg(in[0] + off);
            if (P.nin > 1) {
                const bool ry = (y & (P.part_py - 1)) == 0;
                if (ry) v += __ldg(in[2] + off);
                if ((x & (P.part_px - 1)) == 0) {
                    v += __ldg(in[1] + off);
                    if (ry) v += __ldg(in[3] + off);
                }
            }
        }
        if (QG_IN(r * g.lda + c, g.np * g.lda, 52)) A[r * g.lda + c] = v;
    }
}

// psi = W S_x of one layer into out (interior rows; the wall column x = 0
// gets 0 as in the FFT engines).
__device__ __forceinline__ void store_psi(const SolveParams<float>& P, const float* W,
                                          const float* Sx, float* out, const MtxGeo& g) {
    const int n = g.n, m = g.m;
    const size_t ld = (size_t)P.ld;
    mm3(W, g.lda, Sx, g.ldx, g.mp, g, [&](int r, int c, float v0, float v1) {
        if (r >= n) return;
        float* o = out + (size_t)(r + 1) * ld + 1;
        const long long on = (long long)(P.my + 1) * (long long)ld;
        (void)on;
        if (c < m && QG_IN((long long)(r + 1) * ld + 1 + c, on, 53)) o[c] = v0;
        if (c + 1 < m && QG_IN((long long)(r + 1) * ld + 2 + c, on, 53)) o[c + 1] = v1;
    });
    for (int r = threadIdx.x; r < n; r += kThreads) out[(size_t)(r + 1) * ld] = 0.f;
}

// One solve per CTA: the handle's (BATCH false, one CTA) or member
// blockIdx.x of a batch (one layer), whose fields replace the per-member
// ones of P.  OPY 2: both layers of the two-layer model, with the coupled
// solve of Eqs. isub-1/2 per mode between the transforms.
template <bool BATCH, int OPY>
__global__ void __launch_bounds__(kThreads, 1)
solve_mtx_kernel(SolveParams<float> Pk, const float* __restrict__ tab, MtxGeo g) {
    SolveParams<float> P = Pk;
    if constexpr (BATCH) {
        const SolveMember<float>& M = Pk.batch[blockIdx.x];
#pragma unroll
        for (int q = 0; q < 4; ++q) P.in[0][q] = M.in[q];
        P.nin = M.nin;
        P.part_px = M.part_px;
        P.part_py = M.part_py;
        P.out[0] = M.out;
        P.err = M.err;
    }
    extern __shared__ __align__(16) float sm[];
    __shared__ __align__(8) uint64_t mbar;
    const uint32_t bar = smem_u32(&mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bx = (uint32_t)(g.mp * g.ldx) * 4u, by = (uint32_t)(g.np * g.ldy) * 4u;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"(bx + by) : "memory");
        bulk_copy(smem_u32(sm + g.sx), tab + g.sx, bx, bar);
        bulk_copy(smem_u32(sm + g.sy), tab + g.sy, by, bar);
    }
    pdl_wait();
    pdl_trigger();   // the next fine stage may start staging its own inputs
    float* U = sm + g.u;
    float* V = sm + g.v;
    {
        const float* const in0[4] = {P.in[0][0], P.in[0][1], P.in[0][2], P.in[0][3]};
        load_q(P, in0, U, g);
        if constexpr (OPY == 2) {
            const float* const in1[4] = {P.in[1][0], P.in[1][1], P.in[1][2], P.in[1][3]};
            load_q(P, in1, sm + g.u2, g);
        }
    }
    const bool ok = mbar_wait(bar, 0, kSpin);
    if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) atomicExch(P.err, 1);
        (void)mbar_wait(bar, 0, kSpin);   // let copies in flight land
        return;
    }
    const float* Sx = sm + g.sx;
    const float* Sy = sm + g.sy;
    const int ldb = g.ldb, lda = g.lda;
    const int mp = g.mp;
    auto to_b = [&](float* D) {
        return [D, ldb](int r, int c, float v0, float v1) {
            *reinterpret_cast<float2*>(D + r * ldb + c) = make_float2(v0, v1);
        };
    };
    auto to_a = [&](float* D) {
        return [D, lda](int r, int c, float v0, float v1) {
            *reinterpret_cast<float2*>(D + r * lda + c) = make_float2(v0, v1);
        };
    };
    if constexpr (OPY == 1) {
        // Q S_x -> V (a B operand next)
        mm3(U, lda, Sx, g.ldx, g.mp, g, to_b(V));
        __syncthreads();
        // (S_y Q S_x) o Inv -> U (a B operand next)
        const float* inv = tab + g.tinv;
        mm3(Sy, g.ldy, V, ldb, g.np, g, [&](int r, int c, float v0, float v1) {
            const float2 w = __ldg(reinterpret_cast<const float2*>(inv + r * mp + c));
            *reinterpret_cast<float2*>(U + r * ldb + c) = make_float2(v0 * w.x, v1 * w.y);
        });
        __syncthreads();
        // S_y (...) -> V (an A operand next)
        mm3(Sy, g.ldy, U, ldb, g.np, g, to_a(V));
        __syncthreads();
        // (...) S_x -> psi
        store_psi(P, V, Sx, P.out[0], g);
    } else {
        float* U2 = sm + g.u2;
        float* V2 = sm + g.v2;
        mm3(U, lda, Sx, g.ldx, g.mp, g, to_b(V));
        mm3(U2, lda, Sx, g.ldx, g.mp, g, to_b(V2));
        __syncthreads();
        // the spectra F_i = S_y Q_i S_x of both layers
        mm3(Sy, g.ldy, V, ldb, g.np, g, to_b(U));
        mm3(Sy, g.ldy, V2, ldb, g.np, g, to_b(U2));
        __syncthreads();
        // Eqs. isub-1/2 per mode (k = c + 1, l = r + 1): the 2x2 system with
        // alpha = Ro (lambda_k + lambda_l) (Eq. ialpha), as in the FFT engines
        for (int i = threadIdx.x; i < g.n * g.m; i += kThreads) {
            const int r = i / g.m, c = i - r * g.m;
            const float q1 = P.scale * U[r * ldb + c], q2 = P.scale * U2[r * ldb + c];
            const float al = P.Ro * (__ldg(P.lamx + c + 1) + __ldg(P.lamy + r + 1));
            const float den = al * (al - P.f1 - P.f2);
            U[r * ldb + c] = (al * q1 - P.f2 * q1 - P.f1 * q2) / den;
            U2[r * ldb + c] = (al * q2 - P.f2 * q1 - P.f1 * q2) / den;
        }
        __syncthreads();
        mm3(Sy, g.ldy, U, ldb, g.np, g, to_a(V));
        mm3(Sy, g.ldy, U2, ldb, g.np, g, to_a(V2));
        __syncthreads();
        store_psi(P, V, Sx, P.out[0], g);
        store_psi(P, V2, Sx, P.out[1], g);
    }
}

}  // namespace

size_t mtx_smem_bytes(int mx, int my, int layers) {
    return (size_t)mtx_geo(mx, my, layers).end * sizeof(float);
}

bool mtx_supports(int mx, int my, size_t esz, int layers) {
    return esz == 4 && (layers == 1 || layers == 2) && is_pow2(mx) && is_pow2(my) && mx >= 2 &&
           my >= 2 && mx <= 256 && my <= 256 && mtx_smem_bytes(mx, my, layers) <= 200 * 1024;
}

size_t mtx_table_floats(int mx, int my) { return (size_t)mtx_geo(mx, my).tend; }

void mtx_table(int mx, int my, double dx, double dy, float* out) {
    const MtxGeo g = mtx_geo(mx, my);
    std::fill(out, out + g.tend, 0.0f);
    const double pi = 3.14159265358979323846;
    // sin(pi i k / M) with i k reduced mod 2M first (exact integer argument
    // reduction)
    auto sine = [pi](long ik, int M) { return std::sin(pi * (double)(ik % (2L * M)) / M); };
    for (int i = 0; i < g.m; ++i)
        for (int k = 0; k < g.m; ++k)
            out[g.sx + i * g.ldx + k] = (float)sine((long)(i + 1) * (k + 1), mx);
    for (int j = 0; j < g.n; ++j)
        for (int l = 0; l < g.n; ++l)
            out[g.sy + j * g.ldy + l] = (float)sine((long)(j + 1) * (l + 1), my);
    const double scale = (2.0 / mx) * (2.0 / my);
    for (int l = 0; l < g.n; ++l) {
        const double ly = (2.0 * std::cos(pi * (l + 1) / my) - 2.0) / (dy * dy);
        for (int k = 0; k < g.m; ++k) {
            const double lx = (2.0 * std::cos(pi * (k + 1) / mx) - 2.0) / (dx * dx);
            out[g.tinv + l * g.mp + k] = (float)(scale / (lx + ly));
        }
    }
}

cudaError_t launch_solve_mtx(const SolveParams<float>& P, const float* tab, cudaStream_t s) {
    // (a batch's members carry their own right-hand side planes)
    if (!mtx_supports(P.mx, P.my, sizeof(float), P.layers) || !tab ||
        (!P.batch && (P.nin < 1 || (P.nin > 1 && !(is_pow2(P.part_px) && is_pow2(P.part_py))))))
        return cudaErrorInvalidValue;
    const MtxGeo g = mtx_geo(P.mx, P.my, P.layers);
    const size_t sm = (size_t)g.end * sizeof(float);
    int per = 0, nsm = 0;
    const bool batch = P.batch != nullptr;
    if (batch && (P.nbatch < 1 || P.layers != 1)) return cudaErrorInvalidValue;
    auto k = batch ? solve_mtx_kernel<true, 1>
                   : (P.layers == 2 ? solve_mtx_kernel<false, 2> : solve_mtx_kernel<false, 1>);
    cudaError_t e = launch_shape(reinterpret_cast<const void*>(k), kThreads, sm, &per, &nsm);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(batch ? P.nbatch : 1);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    // allowed to start while the fine stage before it finishes: the table
    // copies precede the programmatic wait, every read of the stage's
    // output follows it
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = P.no_pdl ? nullptr : at;
    cfg.numAttrs = P.no_pdl ? 0 : 1;
    return cudaLaunchKernelEx(&cfg, k, P, tab, g);
}

QG_BOUNDS_QUERY(bounds_site_mtx)

}  // namespace qg
