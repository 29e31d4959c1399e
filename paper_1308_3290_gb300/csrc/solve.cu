// The elliptic sub-problem of Section 4.3 in one cooperative kernel.
//
// Three phases, each a grid-stride loop over pairs of sequences transformed
// by the shared-memory DST-I engine (dst_engine.cuh):
//   1. x pass: rows of the right-hand side (for the one-layer step the
//      restriction arrives as four partial-sum planes, see fused.cu) ->
//      unnormalised DST-I over x (Eq. ifft-1 without its factors), written
//      transposed so phase 2 reads contiguous rows;
//   2. y pass: rows of the transposed array -> DST-I over y, division of mode
//      (k, l) by the eigenvalue of the 5-point Laplacian, lamx[k] + lamy[l],
//      times (2/M_x)(2/M_y) (Eq. ialpha; one layer), or the coupled 2x2
//      solve of Eqs. isub-1/2 with alpha = Ro (lamx + lamy) (two layers: the
//      two layers of a mode form one sequence pair), inverse DST-I over y,
//      written back untransposed;
//   3. x pass: inverse DST-I over x (Eq. ffft-1) -> streamfunction.
// Phases are separated by grid-wide barriers whose waits are bounded (a
// timeout sets the error flag and the kernel returns), and the launch is
// cooperative so that every CTA is resident.  The twiddle tables of both
// directions and the y eigenvalues are bulk-copied into shared memory once.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>

#include "dst_engine.cuh"
#include "qg_internal.cuh"

namespace qg {

cudaError_t launch_shape(const void* kernel, int threads, size_t smem, int* per_sm, int* nsm) {
    struct Key {
        const void* k;
        int threads;
        size_t smem;
        int dev;
        bool operator<(const Key& o) const {
            return std::tie(k, threads, smem, dev) < std::tie(o.k, o.threads, o.smem, o.dev);
        }
    };
    static std::mutex mu;
    static std::map<Key, std::pair<int, int>> cache;
    static std::map<std::pair<const void*, int>, size_t> limit;   // smem limit set per kernel
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const Key key{kernel, threads, smem, dev};
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *per_sm = it->second.first;
            *nsm = it->second.second;
            return cudaSuccess;
        }
    }
    {
        // the limit only ever rises: a launch of a cached shape must still fit
        std::lock_guard<std::mutex> lock(mu);
        size_t& cur = limit[{kernel, dev}];
        if (smem > cur) {
            if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem)) != cudaSuccess)
                return e;
            cur = smem;
        }
    }
    int n = 0, per = 0;
    if ((e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem)) != cudaSuccess)
        return e;
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = {per, n};
    *per_sm = per;
    *nsm = n;
    return cudaSuccess;
}

namespace {

using namespace eng;

constexpr int kMaxThreads = 512;
constexpr int kSpinLimit = 1 << 22;

__host__ __device__ constexpr size_t al16(size_t v) { return (v + 15) / 16 * 16; }

// base-radix butterflies per thread so that a pair of length-N sequences has
// at most kMaxThreads threads, and that pair's thread count (engine E)
__host__ __device__ inline int nb_for(int N, int E) {
    int nb = (2 * N) / (E * kMaxThreads);
    return nb < 1 ? 1 : nb;
}
__host__ __device__ inline int tpr_for(int N, int E) { return (2 * N) / (E * nb_for(N, E)); }
// CTA size of a solve: enough threads for one pair of either direction
__host__ __device__ inline int solve_threads(int mx, int my, int E) {
    int t = tpr_for(mx, E) > tpr_for(my, E) ? tpr_for(mx, E) : tpr_for(my, E);
    return t < 32 ? 32 : t;
}
// complex elements of the sequence buffers of one phase
__host__ __device__ inline size_t bufs_cplx(int N, int threads, int E) {
    return (size_t)(threads / tpr_for(N, E)) * lane_cplx(N);
}

// shared-memory layout (bytes): sequence buffers | lamy | twx | twy
struct Layout {
    size_t lamy, twx, twy, end;
    bool twx_smem, twy_smem;
};
__host__ __device__ inline Layout layout(int mx, int my, size_t esz, int E) {
    Layout L;
    const int th = solve_threads(mx, my, E);
    const size_t cx = 2 * esz;
    const size_t bx = bufs_cplx(mx, th, E), by = bufs_cplx(my, th, E);
    const size_t buf = al16(cx * (bx > by ? bx : by));
    L.twx_smem = 2 * (size_t)mx * cx <= 32 * 1024;
    L.twy_smem = 2 * (size_t)my * cx <= 32 * 1024;
    L.lamy = buf;
    L.twx = al16(L.lamy + esz * (size_t)my);
    L.twy = al16(L.twx + (L.twx_smem ? 2 * (size_t)mx * cx : 0));
    L.end = al16(L.twy + (L.twy_smem ? 2 * (size_t)my * cx : 0));
    return L;
}

// Where the values of a phase's sequence pair come from and go to.
template <typename T>
struct PairIO {
    int N;             // sequence length parameter
    int nrows;         // rows 1..nrows per plane
    int layers;        // planes
    bool pair_planes;  // pair = row r of plane 0 and 1 (else rows r, r+1)
    const T* const* in;  // in[layer * 4 + q]
    int nin, part_px, part_py;
    int ld_in;
    T* const* out;     // out[layer]
    int ld_out;
    bool transpose;
};

// Run one phase: DST-I of every pair (op 0), or DST-I, mode-space solve,
// DST-I (op 1: one layer, op 2: two layers).
template <typename T, int NBM, int E>
__device__ void run_phase(const PairIO<T>& io, int op, CT<T>* bufs, const CT<T>* tw,
                          const T* lamx, const T* slamy, T scale, T Ro, T f1, T f2) {
    const int N = io.N;
    const Geo g = make_geo<E>(N, nb_for(N, E));
    const int lanes = blockDim.x / g.TPR;
    CT<T>* cb = bufs + g.lane * lane_cplx(N);
    const int ppl = io.pair_planes ? io.nrows : (io.nrows + 1) / 2;   // pairs per layer
    const int npairs = io.pair_planes ? ppl : ppl * io.layers;
    const int nslots = (npairs + lanes - 1) / lanes;
    constexpr int EPT = (E / 2) * NBM;  // elements of each sequence per thread (bound)
    const int ept = N / g.TPR;
    for (int slot = blockIdx.x; slot < nslots; slot += gridDim.x) {
        const int pair = slot * lanes + g.lane;
        const bool pv = pair < npairs;
        int la, lb, ra, rb;
        if (io.pair_planes) {
            la = 0;
            lb = 1;
            ra = rb = 1 + pair;
        } else {
            la = lb = pv ? pair / ppl : 0;
            ra = 1 + 2 * (pv ? pair % ppl : 0);
            rb = ra + 1;
        }
        const bool va = pv && ra <= io.nrows, vb = pv && rb <= io.nrows;
        // all loads first
        T av[EPT], bv[EPT];
        const bool rpa = io.nin > 1 && (ra & (io.part_py - 1)) == 0;
        const bool rpb = io.nin > 1 && (rb & (io.part_py - 1)) == 0;
        const T* const* ia = io.in + la * 4;
        const T* const* ib = io.in + lb * 4;
        const size_t oa = (size_t)ra * io.ld_in, ob = (size_t)rb * io.ld_in;
#pragma unroll
        for (int it = 0; it < EPT; ++it) {
            if (it >= ept) break;
            const int j = g.t + it * g.TPR;
            T a = T(0), b = T(0);
            if (j > 0) {
                if (va) a = ia[0][oa + j];
                if (vb) b = ib[0][ob + j];
                if (io.nin > 1) {
                    const bool cx = (j & (io.part_px - 1)) == 0;
                    if (va) {
                        if (cx) a += ia[1][oa + j];
                        if (rpa) a += ia[2][oa + j];
                        if (cx && rpa) a += ia[3][oa + j];
                    }
                    if (vb) {
                        if (cx) b += ib[1][ob + j];
                        if (rpb) b += ib[2][ob + j];
                        if (cx && rpb) b += ib[3][ob + j];
                    }
                }
            }
            av[it] = a;
            bv[it] = b;
        }
#pragma unroll
        for (int it = 0; it < EPT; ++it) {
            if (it >= ept) break;
            put_pair<T>(cb, N, g.t + it * g.TPR, av[it], bv[it]);
        }
        __syncthreads();
        fft_inplace<T, NBM, E>(cb, g, tw);
        if (op != 0) {
            for (int l = g.t; l < N; l += g.TPR) {
                T a = T(0), b = T(0);
                if (l > 0) {
                    const T Fa = dst_a<T>(cb, l);
                    const T Fb = dst_b<T>(cb, l);
                    const T ly = slamy[l];
                    if (op == 1) {
                        if (va) a = Fa * (scale / (lamx[ra] + ly));
                        if (vb) b = Fb * (scale / (lamx[rb] + ly));
                    } else if (va) {
                        const T q1 = scale * Fa, q2 = scale * Fb;
                        const T al = Ro * (lamx[ra] + ly);
                        const T den = al * (al - f1 - f2);
                        a = (al * q1 - f2 * q1 - f1 * q2) / den;
                        b = (al * q2 - f2 * q1 - f1 * q2) / den;
                    }
                }
                put_pair<T>(cb, N, l, a, b);
            }
            __syncthreads();
            fft_inplace<T, NBM, E>(cb, g, tw);
        }
        if (!io.transpose) {
            for (int k = g.t; k < N; k += g.TPR) {
                if (va) io.out[la][(size_t)ra * io.ld_out + k] = (k == 0) ? T(0) : dst_a<T>(cb, k);
                if (vb) io.out[lb][(size_t)rb * io.ld_out + k] = (k == 0) ? T(0) : dst_b<T>(cb, k);
            }
        } else {
            const int nseq = 2 * lanes;
            for (int idx = threadIdx.x; idx < (N - 1) * nseq; idx += blockDim.x) {
                const int c = idx % nseq, k = 1 + idx / nseq;
                const int ln = c >> 1, part = c & 1;
                const int pr = slot * lanes + ln;
                if (pr >= npairs) continue;
                int r, pl;
                if (io.pair_planes) {
                    r = 1 + pr;
                    pl = part;
                } else {
                    r = 1 + 2 * (pr % ppl) + part;
                    pl = pr / ppl;
                }
                if (r > io.nrows) continue;
                const CT<T>* bl = bufs + ln * lane_cplx(N);
                io.out[pl][(size_t)k * io.ld_out + r] = part ? dst_b<T>(bl, k) : dst_a<T>(bl, k);
            }
        }
        __syncthreads();
    }
}

template <typename T, int NBM, int OPY, int E>
__global__ void __launch_bounds__(kMaxThreads)
solve_kernel(SolveParams<T> P) {
    using C = typename Cx<T>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    const Layout Lo = layout(P.mx, P.my, sizeof(T), E);
    C* bufs = reinterpret_cast<C*>(smem);
    T* slamy = reinterpret_cast<T*>(smem + Lo.lamy);
    C* stwx = reinterpret_cast<C*>(smem + Lo.twx);
    C* stwy = reinterpret_cast<C*>(smem + Lo.twy);
    const uint32_t bar = smem_u32(&mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bx = Lo.twx_smem ? (uint32_t)(2 * P.mx * sizeof(C)) : 0u;
        const uint32_t by = Lo.twy_smem ? (uint32_t)(2 * P.my * sizeof(C)) : 0u;
        const uint32_t bl = (uint32_t)(P.my * sizeof(T));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"(bx + by + bl) : "memory");
        if (bx) bulk_copy(smem_u32(stwx), P.twx, bx, bar);
        if (by) bulk_copy(smem_u32(stwy), P.twy, by, bar);
        bulk_copy(smem_u32(slamy), P.lamy, bl, bar);
    }
    pdl_wait();
    pdl_trigger();   // the next fine stage may start staging its own inputs
    const bool ok = mbar_wait(bar, 0, kSpinLimit);
    if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0) atomicExch(P.err, 1);
        (void)mbar_wait(bar, 0, kSpinLimit);     // let copies in flight land
        return;
    }
    const C* twx = Lo.twx_smem ? stwx : P.twx;
    const C* twy = Lo.twy_smem ? stwy : P.twy;
    const bool all = P.split == 0;
    unsigned g0 = grid_gen(P.bar);

    // 1. x pass of the right-hand side, transposed into tr
    if (all || P.phase == 0) {
        PairIO<T> io;
        io.N = P.mx;
        io.nrows = P.my - 1;
        io.layers = P.layers;
        io.pair_planes = false;
        io.in = &P.in[0][0];
        io.nin = P.nin;
        io.part_px = P.part_px;
        io.part_py = P.part_py;
        io.ld_in = P.ld;
        io.out = P.tr;
        io.ld_out = P.ld_tr;
        io.transpose = true;
        run_phase<T, NBM, E>(io, 0, bufs, twx, P.lamx, slamy, P.scale, P.Ro, P.f1, P.f2);
    }
    if (all && !grid_sync(P.bar, P.bar_extra, kSpinLimit, g0)) {
        if (threadIdx.x == 0) atomicExch(P.err, 1);
        return;
    }
    g0 = grid_gen(P.bar);
    // 2. y pass with the mode-space solve, transposed back into work
    if (all || P.phase == 1) {
        const T* trin[8] = {P.tr[0], nullptr, nullptr, nullptr, P.tr[1], nullptr, nullptr, nullptr};
        PairIO<T> io;
        io.N = P.my;
        io.nrows = P.mx - 1;
        io.layers = P.layers;
        io.pair_planes = OPY == 2;
        io.in = trin;
        io.nin = 1;
        io.part_px = io.part_py = 1;
        io.ld_in = P.ld_tr;
        io.out = P.work;
        io.ld_out = P.ld;
        io.transpose = true;
        run_phase<T, NBM, E>(io, OPY, bufs, twy, P.lamx, slamy, P.scale, P.Ro, P.f1, P.f2);
    }
    if (all && !grid_sync(P.bar, P.bar_extra, kSpinLimit, g0)) {
        if (threadIdx.x == 0) atomicExch(P.err, 1);
        return;
    }
    // 3. inverse x pass into out
    if (all || P.phase == 2) {
        const T* win[8] = {P.work[0], nullptr, nullptr, nullptr, P.work[1], nullptr, nullptr, nullptr};
        PairIO<T> io;
        io.N = P.mx;
        io.nrows = P.my - 1;
        io.layers = P.layers;
        io.pair_planes = false;
        io.in = win;
        io.nin = 1;
        io.part_px = io.part_py = 1;
        io.ld_in = P.ld;
        io.out = P.out;
        io.ld_out = P.ld;
        io.transpose = false;
        run_phase<T, NBM, E>(io, 0, bufs, twx, P.lamx, slamy, P.scale, P.Ro, P.f1, P.f2);
    }
}

template <typename T, int NBM, int OPY, int E>
cudaError_t launch_one(const SolveParams<T>& P, size_t sm, cudaStream_t s) {
    auto k = solve_kernel<T, NBM, OPY, E>;
    const int threads = solve_threads(P.mx, P.my, E);
    int nsm = 0, per = 0;
    cudaError_t e = launch_shape(reinterpret_cast<const void*>(k), threads, sm, &per, &nsm);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    // no more CTAs than the largest phase has slots
    auto slots = [threads](int N, int pairs) {
        const int lanes = threads / tpr_for(N, E);
        return (pairs + lanes - 1) / lanes;
    };
    const int ppx = P.layers * (P.my / 2);
    const int ppy = OPY == 2 ? P.mx - 1 : P.mx / 2;
    int want = slots(P.mx, ppx);
    if (slots(P.my, ppy) > want) want = slots(P.my, ppy);
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
        return cudaLaunchKernelEx(&cfg, k, P);
    }
    // one plain launch per pass; stream order separates the passes
    SolveParams<T> Q = P;
    for (int ph = 0; ph < 3; ++ph) {
        Q.phase = ph;
        if ((e = cudaLaunchKernelEx(&cfg, k, Q)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

size_t solve_smem_bytes(int mx, int my, size_t esz, int engine) {
    return layout(mx, my, esz, engine).end;
}

bool solve_engine_supports(int mx, int my, size_t esz, int engine) {
    if (engine == kStreamEngine) return stream_supports(mx, my, esz);
    if (is_warp_engine(engine)) {
        const int rad = warp_engine_radix(engine);
        return solve32_supports(mx, my, rad, esz) &&
               solve32_smem_bytes(mx, my, esz, rad) <= 200 * 1024;
    }
    if (engine != 4 && engine != 16) return false;
    const int nbm = nb_for(mx, engine) > nb_for(my, engine) ? nb_for(mx, engine) : nb_for(my, engine);
    return nbm <= 2 && layout(mx, my, esz, engine).end <= 200 * 1024;
}

template <typename T, int E>
static cudaError_t launch_engine(const SolveParams<T>& P, cudaStream_t s) {
    const size_t sm = layout(P.mx, P.my, sizeof(T), E).end;
    if (sm > 200 * 1024) return cudaErrorInvalidValue;
    const int nbm = nb_for(P.mx, E) > nb_for(P.my, E) ? nb_for(P.mx, E) : nb_for(P.my, E);
    const int opy = P.layers == 2 ? 2 : 1;
    if (nbm <= 1) return opy == 1 ? launch_one<T, 1, 1, E>(P, sm, s) : launch_one<T, 1, 2, E>(P, sm, s);
    if (nbm <= 2) return opy == 1 ? launch_one<T, 2, 1, E>(P, sm, s) : launch_one<T, 2, 2, E>(P, sm, s);
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_solve(const SolveParams<T>& P, int engine, cudaStream_t s) {
    // the partial planes' periods are tested with masks
    if (!P.batch && P.nin > 1 && !(is_pow2(P.part_px) && is_pow2(P.part_py)))
        return cudaErrorInvalidValue;
    if (is_warp_engine(engine)) return launch_solve32<T>(P, warp_engine_radix(engine), s);
    if (engine == kStreamEngine) return launch_solve_stream<T>(P, s);
    if (P.batch) return cudaErrorInvalidValue;   // batches: warp-group engines only
    return engine == 4 ? launch_engine<T, 4>(P, s) : launch_engine<T, 16>(P, s);
}

template cudaError_t launch_solve<float>(const SolveParams<float>&, int, cudaStream_t);
template cudaError_t launch_solve<double>(const SolveParams<double>&, int, cudaStream_t);

}  // namespace qg
