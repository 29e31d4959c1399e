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

#include <cstdint>

#include "bounds.cuh"
#include "dst_engine.cuh"
#include "solve_mtx.h"

namespace qg {
namespace {

using namespace eng;

constexpr int kThreads = 128;   // = the MMA's M: one thread per row
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
// 16 consecutive TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t ta, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Layout of one grid (bytes of shared memory): mp, np the interior sizes
// rounded up to 16 (x and y).  Operands (hi then lo halves, each `half`
// bytes apart):
//   SX: B operand of products 1 and 4, mp rows x K = mp;
//   SY: A operand of products 2 and 3, 128 rows x K = np (rows >= np zero);
//   OP: A operand of products 1 and 4 (128 rows x K = mp, rows >= np zero)
//       or B operand of products 2 and 3 (mp rows x K = np).
struct TcGeo {
    int m, n, mp, np;
    int sx, sx_half, sy, sy_half, op, op_half, end;
    int cols;   // TMEM columns (a power of two >= 32)
    int ldx, ldy, sxg, syg, ting;   // the engine-40 table: pitches and offsets (floats)
};
__host__ __device__ inline int r16(int v) { return (v + 15) / 16 * 16; }
__host__ __device__ inline TcGeo tc_geo(int mx, int my) {
    TcGeo g;
    g.m = mx - 1;
    g.n = my - 1;
    g.mp = r16(g.m);
    g.np = r16(g.n);
    g.sx_half = g.mp * g.mp * 4;
    g.sy_half = kThreads * g.np * 4;
    const int opa = kThreads * g.mp * 4, opb = g.mp * g.np * 4;
    g.op_half = opa > opb ? opa : opb;
    g.sx = 0;
    g.sy = g.sx + 2 * g.sx_half;
    g.op = g.sy + 2 * g.sy_half;
    g.end = g.op + 2 * g.op_half;
    const int c1 = (g.mp / 8) * g.mp, c2 = (g.np / 8) * g.mp;   // k-steps x N
    const int c = c1 > c2 ? c1 : c2;
    g.cols = 32;
    while (g.cols < c) g.cols *= 2;
    // the engine-40 table (solve_mtx.cu's layout): S_x | S_y | Inv
    g.ldx = g.mp + 8;
    g.ldy = g.np + 4;
    g.sxg = 0;
    g.syg = g.mp * g.ldx;
    g.ting = g.syg + g.np * g.ldy;   // Inv: np x mp, pitch mp
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
// accumulators of N columns each, issued by thread 0 and committed to bar.
__device__ __forceinline__ void issue(uint32_t taddr, uint32_t a, int a_half, uint32_t b,
                                      int b_half, int N, int K, uint32_t bar) {
    const uint32_t id = idesc_tf32(kThreads, N);
    const uint32_t sboa = (uint32_t)(K / 4) * 128u, sbob = sboa;
    for (int ks = 0; ks < K / 8; ++ks) {
        const uint32_t o = (uint32_t)ks * 256u;
        const uint32_t d = taddr + (uint32_t)(ks * N);
        const uint64_t ah = sdesc(a + o, 128, sboa), al = sdesc(a + a_half + o, 128, sboa);
        const uint64_t bh = sdesc(b + o, 128, sbob), bl = sdesc(b + b_half + o, 128, sbob);
        mma_tf32(d, al, bh, id, 0);
        mma_tf32(d, ah, bl, id, 1);
        mma_tf32(d, ah, bh, id, 1);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(bar) : "memory");
}

// Row `lane row` of a product: the sum of its K/8 accumulators, N <= 64.
__device__ __forceinline__ void row_sum(uint32_t taddr, int N, int K, float (&out)[64]) {
    const uint32_t lane = (uint32_t)(threadIdx.x & ~31) << 16;
#pragma unroll
    for (int j = 0; j < 64; ++j) out[j] = 0.f;
    for (int ks = 0; ks < K / 8; ++ks) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (16 * c >= N) break;
            float v[16];
            tmem_ld16(taddr + lane + (uint32_t)(ks * N + 16 * c), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) out[16 * c + j] += v[j];
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
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_taddr;
    const int i = threadIdx.x;
    const uint32_t bar = smem_u32(&mbar);
    const uint32_t base = smem_u32(sm);
    if (i == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the constant operands (before the programmatic wait): zero the padded
    // arrays, then S_x (B, N = mp rows) and S_y (A, rows < np) split
    for (int o = 4 * i; o < g.end; o += 4 * kThreads)
        *reinterpret_cast<uint32_t*>(sm + o) = 0u;
    __syncthreads();
    for (int e = i; e < g.mp * g.mp; e += kThreads) {
        const int r = e / g.mp, k = e - r * g.mp;
        const float v = (r < g.m && k < g.m) ? __ldg(tab + g.sxg + r * g.ldx + k) : 0.f;
        put_split(sm + g.sx, g.sx_half, kmaj(r, k, g.mp), v, 2 * g.sx_half);
    }
    for (int e = i; e < g.np * g.np; e += kThreads) {
        const int r = e / g.np, k = e - r * g.np;
        const float v = (r < g.n && k < g.n) ? __ldg(tab + g.syg + r * g.ldy + k) : 0.f;
        put_split(sm + g.sy, g.sy_half, kmaj(r, k, g.np), v, 2 * g.sy_half);
    }
    if (i < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&s_taddr)), "r"(g.cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    pdl_wait();
    pdl_trigger();   // the next fine stage may start staging its own inputs
    // Q (A operand of product 1): row i = y - 1, column x - 1, the sum of the
    // restriction's partial planes as in the FFT engines
    if (i < g.n) {
        const int y = i + 1;
        const bool ry = P.nin > 1 && y % P.part_py == 0;
        for (int c = 0; c < g.m; ++c) {
            const int x = c + 1;
            const size_t off = (size_t)y * P.ld + x;
            float v = 0.f;
            if (QG_IN((long long)off, (long long)(P.my + 1) * P.ld, 82)) {
                v = __ldg(P.in[0][0] + off);
                if (P.nin > 1) {
                    if (ry) v += __ldg(P.in[0][2] + off);
                    if (x % P.part_px == 0) {
                        v += __ldg(P.in[0][1] + off);
                        if (ry) v += __ldg(P.in[0][3] + off);
                    }
                }
            }
            put_split(sm + g.op, g.op_half, kmaj(i, c, g.mp), v, 2 * g.op_half);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t taddr = s_taddr;
    const uint32_t sx = base + g.sx, sy = base + g.sy, op = base + g.op;
    int ok = 1;
    float row[64];
    for (int step = 0; step < 4; ++step) {
        // products 1, 4: (OP as A) (S_x as B), K = mp; 2, 3: (S_y as A) (OP as B), K = np
        const bool xs = step == 0 || step == 3;
        const int K = xs ? g.mp : g.np;
        if (i == 0 && ok) {
            if (xs) issue(taddr, op, g.op_half, sx, g.sx_half, g.mp, K, bar);
            else issue(taddr, sy, g.sy_half, op, g.op_half, g.mp, K, bar);
        }
        ok = ok && mbar_wait(bar, (uint32_t)(step & 1), kSpin) ? 1 : 0;
        if (!__syncthreads_and(ok)) {
            ok = 0;
            break;
        }
        fence_after();
        row_sum(taddr, g.mp, K, row);
        fence_before();
        __syncthreads();   // every read of the operands and of TMEM is done
        if (step == 3) break;
        if (i < g.n) {
            if (step == 1) {
                const float* inv = tab + g.ting + i * g.mp;
#pragma unroll
                for (int c = 0; c < 64; ++c)
                    if (c < g.mp) row[c] *= __ldg(inv + c);
            }
            if (step == 2) {
                // W = S_y U as the A operand of product 4: row i
#pragma unroll
                for (int c = 0; c < 64; ++c)
                    if (c < g.mp) put_split(sm + g.op, g.op_half, kmaj(i, c, g.mp), row[c],
                                            2 * g.op_half);
            } else {
                // V (product 1) or U (product 2) transposed as the B operand of
                // the next product: column i of the mp x np operand
#pragma unroll
                for (int c = 0; c < 64; ++c)
                    if (c < g.mp) put_split(sm + g.op, g.op_half, kmaj(c, i, g.np), row[c],
                                            2 * g.op_half);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        fence_after();
    }
    if (!ok) {
        if (i == 0) atomicExch(P.err, 1);
    } else if (i < g.n) {
        // psi at interior row y = i + 1; the wall column x = 0 gets 0 as in
        // the FFT engines
        float* o = P.out[0] + (size_t)(i + 1) * P.ld;
        const long long on = (long long)(P.my + 1) * P.ld;
        (void)on;
        if (QG_IN((long long)(i + 1) * P.ld, on, 83)) o[0] = 0.f;
#pragma unroll
        for (int c = 0; c < 64; ++c)
            if (c < g.m && QG_IN((long long)(i + 1) * P.ld + 1 + c, on, 83)) o[1 + c] = row[c];
    }
    fence_before();
    __syncthreads();
    if (i < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                     "r"(g.cols) : "memory");
}

}  // namespace

bool tc_supports(int mx, int my, size_t esz, int layers) {
    return esz == 4 && layers == 1 && is_pow2(mx) && is_pow2(my) && mx >= 16 && my >= 16 &&
           mx <= 64 && my <= 64;
}

cudaError_t launch_solve_tc(const SolveParams<float>& P, const float* tab, cudaStream_t s) {
    if (!tc_supports(P.mx, P.my, sizeof(float), P.layers) || !tab ||
        (!P.batch && (P.nin < 1 || (P.nin > 1 && (P.part_px < 1 || P.part_py < 1)))))
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
