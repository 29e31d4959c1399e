// Elliptic solve of Section 4.3 in matrix form on the fifth-generation
// tensor cores (engine 41): tcgen05.mma with TMEM accumulators, for small
// one-layer FP32 grids (sides of 16, 32 or 64 intervals).
//
// The same four products as the matrix form of solve_mtx.cu (engine 40),
//
//     V = Q S_x,  U = (S_y V) o Inv,  W = S_y U,  Psi = W S_x,
//
// with the sine matrices S_x[i][k] = sin(pi i k / Mx), S_y[j][l] =
// sin(pi j l / My) and Inv = (2/Mx)(2/My)/lambda (Eqs. ffft-1, ialpha,
// ifft-1), and the same precision scheme: every FP32 operand x is split into
// TF32 numbers hi = rn(x), lo = rn(x - hi), and each k-step (8 terms of the
// sum) is lo*hi + hi*lo + hi*hi accumulated from zero, the small terms
// first; the k-steps are summed with round-to-nearest FP32 adds.  (The
// tensor core's accumulation truncates: fed the running sum, it shrinks
// every output by about 2^-23 per k-step.)  Here each k-step has an
// accumulator of its own in TMEM, so one product is K/8 x 3 tcgen05.mma
// instructions issued by one thread and completed by one tcgen05.commit.
//
// One CTA of 128 threads per grid (the handle's, or one per ensemble
// member): thread i owns row i of the 128-row tile (rows beyond the grid's
// are zero), reads its row of each result from TMEM lane i
// (tcgen05.ld.32x32b), sums the k-step accumulators, and writes the row
// into shared memory as the next product's operand: as an A operand
// (K-major, row i) or transposed as a B operand (column i).  Operands are
// K-major without swizzle: 8 x 16-byte core matrices, 128 bytes apart along
// K (LBO) and K/4 x 128 bytes apart along M or N (SBO).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "bounds.cuh"
#include "dst_engine.cuh"
#include "solve_mtx.h"

namespace qg {
namespace {

using namespace eng;

constexpr int kM = 128;         // the MMA's M: rows of every product
constexpr int kThreads = 256;  // two warps per 32-lane TMEM group: each reads half the columns
constexpr int kSpin = 1 << 22;

__device__ __forceinline__ uint32_t tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Byte offset of element (r, k) of a K-major operand with K columns.
__host__ __device__ constexpr int kmaj(int r, int k, int K) {
    return (r >> 3) * (K / 4) * 128 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

// Shared-memory matrix descriptor: K-major, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of this architecture
    return d;
}
// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t id, int acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                 ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
}
__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 8 consecutive TMEM columns of this thread's lane (no wait)
__device__ __forceinline__ void tmem_ld8(uint32_t ta, uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(ta));
}
__device__ __forceinline__ void tmem_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Layout of one grid (bytes of shared memory): mp, np the interior sizes
// rounded up to 16 (x and y).  Operands (hi then lo halves, each `half`
// bytes apart):
//   SX: B operand of products 1 and 4, mp rows x K = mp;
//   SY: A operand of products 2 and 3, 128 rows x K = np (rows >= np zero);
//   OP: A operand of products 1 and 4 (128 rows x K = mp) or B operand of
//       products 2 and 3 (mp rows x K = np).
// SX and SY come ready-made (split, zero-padded, in this layout) from the
// grid's table (tc_table), followed there by Inv (np x mp floats).
struct TcGeo {
    int m, n, mp, np;
    int sx, sx_half, sy, sy_half, op, op_half, end;
    int cols;      // TMEM columns (a power of two >= 32)
    int tab_inv;   // floats before Inv in the table
};
__host__ __device__ inline int r16(int v) { return (v + 15) / 16 * 16; }
__host__ __device__ inline TcGeo tc_geo(int mx, int my) {
    TcGeo g;
    g.m = mx - 1;
    g.n = my - 1;
    g.mp = r16(g.m);
    g.np = r16(g.n);
    g.sx_half = g.mp * g.mp * 4;
    g.sy_half = kM * g.np * 4;
    const int opa = kM * g.mp * 4, opb = g.mp * g.np * 4;
    g.op_half = opa > opb ? opa : opb;
    g.sx = 0;
    g.sy = g.sx + 2 * g.sx_half;
    g.op = g.sy + 2 * g.sy_half;
    g.end = g.op + 2 * g.op_half;
    const int c1 = (g.mp / 8) * g.mp, c2 = (g.np / 8) * g.mp;   // k-steps x N
    const int c = c1 > c2 ? c1 : c2;
    g.cols = 32;
    while (g.cols < c) g.cols *= 2;
    g.tab_inv = g.op / 4;
    return g;
}

// Store x split as (hi, lo) at byte offset off of an operand.
__device__ __forceinline__ void put_split(unsigned char* base, int half, int off, float x,
                                          int lim) {
    (void)lim;
    if (!QG_IN(off + half, lim, 81)) return;
    const uint32_t hi = tf32_rn(x);
    const uint32_t lo = tf32_rn(x - __uint_as_float(hi));
    *reinterpret_cast<uint32_t*>(base + off) = hi;
    *reinterpret_cast<uint32_t*>(base + off + half) = lo;
}

// One product D = A B^T (A: 128 x K, B: N x K, both split) into K/8
// accumulators of N columns each, issued by one thread and committed to bar.
__device__ __forceinline__ void issue(uint32_t taddr, uint32_t a, int a_half, uint32_t b,
                                      int b_half, int N, int K, uint32_t bar) {
    const uint32_t id = idesc_tf32(kM, N);
    const uint32_t sbo = (uint32_t)(K / 4) * 128u;
    for (int ks = 0; ks < K / 8; ++ks) {
        const uint32_t o = (uint32_t)ks * 256u;
        const uint32_t d = taddr + (uint32_t)(ks * N);
        const uint64_t ah = sdesc(a + o, 128, sbo), al = sdesc(a + a_half + o, 128, sbo);
        const uint64_t bh = sdesc(b + o, 128, sbo), bl = sdesc(b + b_half + o, 128, sbo);
        mma_tf32(d, al, bh, id, 0);
        mma_tf32(d, ah, bl, id, 1);
        mma_tf32(d, ah, bh, id, 1);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(bar) : "memory");
}

// This thread's part of a product's row: columns c0 .. c0 + N/2 - 1 of TMEM
// lane `lane`, the sum of the K/8 accumulators (round-to-nearest adds).
__device__ __forceinline__ void row_sum(uint32_t taddr, uint32_t lane, int c0, int N, int K,
                                        float (&out)[32]) {
#pragma unroll
    for (int j = 0; j < 32; ++j) out[j] = 0.f;
    const int nh = N / 2;
    for (int ks = 0; ks < K / 8; ++ks) {
        uint32_t r[4][8];
        const uint32_t ta = taddr + lane + (uint32_t)(ks * N + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (8 * q < nh) tmem_ld8(ta + 8 * q, r[q]);
        tmem_wait();
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (8 * q < nh) {
#pragma unroll
                for (int j = 0; j < 8; ++j) out[8 * q + j] += __uint_as_float(r[q][j]);
            }
    }
}

// One solve per CTA: the handle's (BATCH false) or member blockIdx.x of a
// batch, whose fields replace the per-member ones of P.
template <bool BATCH>
__global__ void __launch_bounds__(kThreads, 1)
solve_tc_kernel(SolveParams<float> Pk, const float* __restrict__ tab, TcGeo g) {
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
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mb_tab, mb_mma;
    __shared__ uint32_t s_taddr;
    const int t = threadIdx.x, w = t >> 5;
    const int row = 32 * (w & 3) + (t & 31);      // TMEM lane = row of the products
    const int half = w >> 2;                      // which half of the columns
    const uint32_t lane = (uint32_t)(32 * (w & 3)) << 16;
    const uint32_t btab = smem_u32(&mb_tab), bmma = smem_u32(&mb_mma);
    const uint32_t base = smem_u32(sm);
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(btab) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bmma) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // the split sine matrices, ready-made in the table (constants: copied
    // before the programmatic wait)
    const uint32_t tab_bytes = (uint32_t)g.op;
    if (t == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(btab),
                     "r"(tab_bytes) : "memory");
        bulk_copy(base, tab, tab_bytes, btab);
    }
    // OP starts zero (rows and columns beyond the grid's)
    for (int o = 16 * t; o < 2 * g.op_half; o += 16 * kThreads)
        *reinterpret_cast<uint4*>(sm + g.op + o) = make_uint4(0u, 0u, 0u, 0u);
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&s_taddr)), "r"(g.cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    pdl_wait();
    pdl_trigger();   // the next fine stage may start staging its own inputs
    // Q (A operand of product 1, row r = y - 1, column c = x - 1): the sum of
    // the restriction's partial planes as in the FFT engines
    for (int e = t; e < g.n * g.mp; e += kThreads) {
        const int r = e / g.mp, c = e - r * g.mp;
        const int y = r + 1, x = c + 1;
        float v = 0.f;
        const size_t off = (size_t)y * P.ld + x;
        if (c < g.m && QG_IN((long long)off, (long long)(P.my + 1) * P.ld, 82)) {
            v = __ldg(P.in[0][0] + off);
            if (P.nin > 1) {
                const bool ry = (y & (P.part_py - 1)) == 0;
                if (ry) v += __ldg(P.in[0][2] + off);
                if ((x & (P.part_px - 1)) == 0) {
                    v += __ldg(P.in[0][1] + off);
                    if (ry) v += __ldg(P.in[0][3] + off);
                }
            }
        }
        put_split(sm + g.op, g.op_half, kmaj(r, c, g.mp), v, 2 * g.op_half);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    int ok = mbar_wait(btab, 0, kSpin) ? 1 : 0;
    fence_before();
    ok = __syncthreads_and(ok);
    fence_after();
    const uint32_t taddr = s_taddr;
    const uint32_t sx = base + g.sx, sy = base + g.sy, op = base + g.op;
    const int nh = g.mp / 2, c0 = half * nh;
    float acc[32];
    for (int step = 0; step < 4 && ok; ++step) {
        // products 1, 4: (OP as A) (S_x as B), K = mp; 2, 3: (S_y as A) (OP as B), K = np
        const bool xs = step == 0 || step == 3;
        const int K = xs ? g.mp : g.np;
        if (t == 0) {
            if (xs) issue(taddr, op, g.op_half, sx, g.sx_half, g.mp, K, bmma);
            else issue(taddr, sy, g.sy_half, op, g.op_half, g.mp, K, bmma);
        }
        ok = mbar_wait(bmma, (uint32_t)(step & 1), kSpin) ? 1 : 0;
        if (!__syncthreads_and(ok)) {
            ok = 0;
            break;
        }
        fence_after();
        row_sum(taddr, lane, c0, g.mp, K, acc);
        fence_before();
        __syncthreads();   // every read of the operands and of TMEM is done
        if (step == 3) break;
        if (row < g.n) {
            if (step == 1) {
                const float* inv = tab + g.tab_inv + row * g.mp + c0;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < nh) acc[j] *= __ldg(inv + j);
            }
            if (step == 2) {
                // W = S_y U as the A operand of product 4: row `row`
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < nh) put_split(sm + g.op, g.op_half, kmaj(row, c0 + j, g.mp), acc[j],
                                          2 * g.op_half);
            } else {
                // V (product 1) or U (product 2) transposed as the B operand of
                // the next product: column `row` of the mp x np operand
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < nh) put_split(sm + g.op, g.op_half, kmaj(c0 + j, row, g.np), acc[j],
                                          2 * g.op_half);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        fence_after();
    }
    if (!ok) {
        if (t == 0) atomicExch(P.err, 1);
    } else if (row < g.n) {
        // psi at interior row y = row + 1; the wall column x = 0 gets 0 as in
        // the FFT engines
        float* o = P.out[0] + (size_t)(row + 1) * P.ld;
        const long long on = (long long)(P.my + 1) * P.ld;
        (void)on;
        if (half == 0 && QG_IN((long long)(row + 1) * P.ld, on, 83)) o[0] = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < nh && c0 + j < g.m && QG_IN((long long)(row + 1) * P.ld + 1 + c0 + j, on, 83))
                o[1 + c0 + j] = acc[j];
    }
    fence_before();
    __syncthreads();
    if (w == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                     "r"(g.cols) : "memory");
}

// Round to nearest TF32, ties away from zero (the device's cvt.rna.tf32).
float rna_tf32(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    b = (b + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

}  // namespace

bool tc_supports(int mx, int my, size_t esz, int layers) {
    return esz == 4 && layers == 1 && is_pow2(mx) && is_pow2(my) && mx >= 16 && my >= 16 &&
           mx <= 64 && my <= 64;
}

size_t tc_table_floats(int mx, int my) {
    const TcGeo g = tc_geo(mx, my);
    return (size_t)g.tab_inv + (size_t)g.np * g.mp;
}

void tc_table(int mx, int my, double dx, double dy, float* out) {
    const TcGeo g = tc_geo(mx, my);
    std::fill(out, out + tc_table_floats(mx, my), 0.0f);
    const double pi = 3.14159265358979323846;
    // sin(pi i k / M) with i k reduced mod 2M first (exact integer argument
    // reduction), split as hi = rn_tf32(s), lo = rn_tf32(s - hi)
    auto put = [&](int off_bytes, int half_bytes, double v) {
        const float s = (float)v;
        const float hi = rna_tf32(s);
        out[off_bytes / 4] = hi;
        out[(off_bytes + half_bytes) / 4] = rna_tf32(s - hi);
    };
    auto sine = [pi](long ik, int M) { return std::sin(pi * (double)(ik % (2L * M)) / M); };
    for (int i = 0; i < g.m; ++i)
        for (int k = 0; k < g.m; ++k)
            put(g.sx + kmaj(i, k, g.mp), g.sx_half, sine((long)(i + 1) * (k + 1), mx));
    for (int j = 0; j < g.n; ++j)
        for (int l = 0; l < g.n; ++l)
            put(g.sy + kmaj(j, l, g.np), g.sy_half, sine((long)(j + 1) * (l + 1), my));
    const double scale = (2.0 / mx) * (2.0 / my);
    for (int l = 0; l < g.n; ++l) {
        const double ly = (2.0 * std::cos(pi * (l + 1) / my) - 2.0) / (dy * dy);
        for (int k = 0; k < g.m; ++k) {
            const double lx = (2.0 * std::cos(pi * (k + 1) / mx) - 2.0) / (dx * dx);
            out[g.tab_inv + l * g.mp + k] = (float)(scale / (lx + ly));
        }
    }
}

cudaError_t launch_solve_tc(const SolveParams<float>& P, const float* tab, cudaStream_t s) {
    if (!tc_supports(P.mx, P.my, sizeof(float), P.layers) || !tab ||
        (!P.batch && (P.nin < 1 || (P.nin > 1 && !(is_pow2(P.part_px) && is_pow2(P.part_py))))))
        return cudaErrorInvalidValue;
    const bool batch = P.batch != nullptr;
    if (batch && P.nbatch < 1) return cudaErrorInvalidValue;
    const TcGeo g = tc_geo(P.mx, P.my);
    auto k = batch ? solve_tc_kernel<true> : solve_tc_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, g.end);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(batch ? P.nbatch : 1);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = (size_t)g.end;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = P.no_pdl ? nullptr : at;
    cfg.numAttrs = P.no_pdl ? 0 : 1;
    return cudaLaunchKernelEx(&cfg, k, P, tab, g);
}

QG_BOUNDS_QUERY(bounds_site_tc)

}  // namespace qg
