// C-ABI of libqgcgp: handle management, tables, and the CGPRK3 step.
//
// The step (Section 3.2) is TVDRK3 (Section 4.2) in which every stage
//   (ii)  restricts the fine state to the elliptic grid (Eq. res, l times),
//   (iii) solves the elliptic sub-problem there with the sine-transform
//         solver (Eqs. ifft-1, ialpha, ffft-1; Eqs. isub-1/2 for 2 layers),
//   (iv)  prolongs the streamfunction back (Eq. pro, l times),
//   (i)   and updates the fine state with the stage's right-hand side.
// The kernels of one step are captured once into a CUDA graph and replayed.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <type_traits>
#include <vector>

#include "qg_internal.cuh"
#include "solve_mtx.h"

namespace {
// NVTX range around a public call (shown by Nsight Systems and by
// ncu --nvtx); the header-only NVTX 3 API costs nothing without a tool.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

using namespace qg;

namespace {

struct LevelTables {
    int mx = 0, my = 0, ldc = 0;
    double dxc = 0, dyc = 0;
    void* twx = nullptr;   // e^{i pi t/mx}, t < 2 mx   (Cx<T>)
    void* twy = nullptr;   // e^{i pi t/my}, t < 2 my
    void* lamx = nullptr;  // (2 cos(pi k/mx) - 2)/dxc^2, k = 0..mx
    void* lamy = nullptr;  // (2 cos(pi l/my) - 2)/dyc^2, l = 0..my
    void* ptx[3] = {nullptr, nullptr, nullptr};  // warp-group engine pass twiddles for
    void* pty[3] = {nullptr, nullptr, nullptr};  //   L = 2 mx and 2 my, engines 32/33/34
    void* mtab = nullptr;  // matrix engine (FP32, one layer): sine matrices and 1/lambda
    void* tctab = nullptr; // engine 41: split sine matrices (shared-memory image), 1/lambda
};

// Multigrid hierarchy below one elliptic grid (multigrid.cu): grids 1..nl-1
// (grid 0 is the caller's psi; rhs[0] holds its summed right-hand side),
// each psi and rhs with (my + 1) rows of pitch ld and zero walls.
struct MGPlan {
    int nl = 0, tail = 0;
    std::vector<int> mx, my, ld;
    std::vector<void*> psi, rhs;
};

}  // namespace

// Forward states kept for the adjoint (one layer): the state at every
// `every`-th step, the states of the segment being reversed (every > 1), the
// handle's state when the reversal began, and the adjoint's work fields.
struct Tape {
    int64_t every = 1, max_steps = 0, recorded = 0, cursor = 0;
    bool reversing = false;
    std::vector<void*> ckpt;
    std::vector<void*> seg;
    int64_t seg_start = -1;
    void* live = nullptr;
    enum { W1, W2, P0, P1, P2, U, PHI, L0, L1, ACC, GF, NBUF };
    void* buf[NBUF] = {};
    std::vector<void*> allocs;
};

struct qg_ctx {
    int layers = 1;
    qg_dtype dtype = QG_F32;
    size_t esz = 4;
    int nx = 0, ny = 0, levels = 0;
    double x0 = 0, x1 = 1, y0 = -1, y1 = 1, dx = 0, dy = 0;
    double Re = 0, Ro = 0, Fr = 0, delta = 0, sigma = 0, dt = 0, amp = 1;
    int ldf = 0;
    size_t plane_f = 0;            // elements of one fine plane
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;    // private stream used for graph capture
    cudaStream_t side = nullptr;   // two layers: the second layer's fine stage branch
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    void* w[3] = {nullptr, nullptr, nullptr};  // w^n, w^(1), w^(2) (layers planes each)
    void* psi = nullptr;           // fine psi (layers planes)
    void* cw = nullptr;            // elliptic-grid work (layers planes)
    void* cpsi = nullptr;          // elliptic-grid psi (layers planes)
    size_t plane_c = 0;
    void* ct = nullptr;            // transposed x-spectrum of the elliptic grid (layers planes)
    int ld_t = 0;                  // its pitch (round_up(my + 1, 32))
    size_t plane_t = 0;            // its plane size ((mx + 1) rows)
    void* part = nullptr;          // 4 restriction partial-sum planes (one layer, l >= 1)
    bool part_valid = false;       // part holds R^l w^n of the current state
    void* frow = nullptr;          // forcing per fine row
    void* f2d = nullptr;           // forcing field in use (padded fine) or null
    void* f2d_buf = nullptr;       // its storage, allocated on first use
    std::map<int, LevelTables> tables;
    std::map<int, void*> twcache;
    double* dpart = nullptr;
    double* dout = nullptr;
    double* hout = nullptr;        // pinned host copy of the 5 diagnostics
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    qg_status latched = QG_OK;
    std::vector<void*> allocs;
    size_t alloc_bytes = 0;        // device bytes held through dev_alloc
    // per-kernel timing (bench instrumentation): events recorded in the graph
    bool timing = false;
    unsigned timing_mask = ~0u;    // kernel classes bracketed by timing events
    int fault = QG_FAULT_NONE;     // failure-detection test switch
    uint64_t graph_gen = 0;        // bumped whenever the captured step is invalidated
    bool split_solve = false;      // solve as three plain launches (ensemble
                                   // members: no cooperative grids side by side)
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
    size_t ev_next = 0;
    int64_t kernels_per_step = 0;
    bool capturing = false;
    // TMA tensor maps of the fine buffers (halo and interior boxes)
    // (per layer: [k][layer]; the second layer's maps exist for two layers)
    CUtensorMap tm_halo[3][2], tm_int[3][2], tm_psi, tm_f;
    int solve_engine = 4;          // FFT base radix of the step's solve (autotuned)
    bool engine_forced = false;    // solve_engine was forced by QG_SOLVE_ENGINE
    int fine_rows = 0;             // fine rows per CTA of the fused stage (autotuned)
    int fine_ry = 8;               // fine rows each of its threads sweeps (autotuned)
    // transfers with pinned host memory (qg_set_state, qg_get_state_async):
    // DMA on two internal streams through device staging buffers (two per
    // direction, dense exchange layout), ordered against the handle's
    // stream by events, so that they overlap the steps around them
    cudaStream_t xin = nullptr, xout = nullptr;
    void* stage_in[2] = {nullptr, nullptr};
    void* stage_out[2] = {nullptr, nullptr};
    cudaEvent_t in_ready[2] = {}, in_free[2] = {}, out_ready[2] = {}, out_free[2] = {};
    int bin = 0, bout = 0;
    bool member = false;           // an ensemble member (keeps the default tile)
    int* derr = nullptr;           // device error flag of bounded waits
    unsigned* dbar = nullptr;      // grid-barrier counters of the solve kernel
    Tape* tape = nullptr;          // adjoint tape (qg_tape_begin .. qg_tape_end)
    double cfl = 0.0;              // > 0: adaptive step (Eq. dt) with this CFL number
    double time_host = 0.0;        // model time of two-layer handles (fixed dt)
    bool stats = false;            // accumulate the first-stage psi of every step
    double* stat_acc = nullptr;    // its FP64 sum (elliptic grid, or fine for l = 0 / 2 layers)
    double* stat_acc_w = nullptr;  // FP64 sum of the state w^n (fine, layers planes)
    int64_t stat_count = 0;
    double* dclock = nullptr;      // device {umax bits, time, last dt, spare}
    int solver = QG_SOLVER_FFT;    // elliptic solver of the step and qg_poisson_solve
    int mg_cycles = 4;             // V-cycles per multigrid solve
    std::map<long, MGPlan> mg;     // multigrid hierarchies by (mx, my)
};

namespace qg {

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

cudaError_t make_tensor_map(CUtensorMap* m, const void* base, int nx, int ny, int ld,
                            size_t esz, int bw, int bh) {
    auto fn = tensor_map_encoder();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)nx + 1, (cuuint64_t)ny + 1};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * esz};
    const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = fn(m, esz == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                          2, const_cast<void*>(base), dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace qg

namespace {

qg_status fail(qg_ctx* h, qg_status s) {
    if (h && h->latched == QG_OK) h->latched = s;
    return s;
}

qg_status cuda_status(qg_ctx* h, cudaError_t e) {
    if (e == cudaSuccess) return QG_OK;
    if (e == cudaErrorMemoryAllocation) return fail(h, QG_ERR_OOM);
    return fail(h, QG_ERR_CUDA);
}

#define QG_TRY(expr)                                \
    do {                                            \
        cudaError_t e_ = (expr);                    \
        if (e_ != cudaSuccess) return cuda_status(h, e_); \
    } while (0)

// A call returning qg_status: latch and return its error.
#define QG_TRY_S(expr)                              \
    do {                                            \
        const qg_status st_ = (expr);               \
        if (st_ != QG_OK) return fail(h, st_);      \
    } while (0)

// QG_ALLOC_LIMIT_BYTES (a test hook for the out-of-memory path): the device
// bytes one handle may hold; an allocation past it fails as a failed
// cudaMalloc does, with QG_ERR_OOM.
qg_status dev_alloc(qg_ctx* h, void** p, size_t bytes) {
    if (const char* lim = std::getenv("QG_ALLOC_LIMIT_BYTES")) {
        const unsigned long long cap = std::strtoull(lim, nullptr, 10);
        if (cap > 0 && h->alloc_bytes + bytes > cap) {
            *p = nullptr;
            return QG_ERR_OOM;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        (void)cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? QG_ERR_OOM : QG_ERR_CUDA;
    }
    h->allocs.push_back(*p);
    h->alloc_bytes += bytes;
    e = cudaMemset(*p, 0, bytes);
    return e == cudaSuccess ? QG_OK : QG_ERR_CUDA;
}

int padded_ld(int n) { return round_up(n + 1, 32); }

// Twiddle table tw[t] = e^{i pi t / N}, t = 0..2N-1, generated in FP64.
qg_status get_twiddles(qg_ctx* h, int N, void** out) {
    auto it = h->twcache.find(N);
    if (it != h->twcache.end()) {
        *out = it->second;
        return QG_OK;
    }
    const size_t n = 2 * (size_t)N;
    void* d = nullptr;
    qg_status s = dev_alloc(h, &d, n * 2 * h->esz);
    if (s != QG_OK) return s;
    const double pi = 3.14159265358979323846;
    if (h->dtype == QG_F64) {
        std::vector<double> t(2 * n);
        for (size_t k = 0; k < n; ++k) {
            t[2 * k] = std::cos(pi * (double)k / N);
            t[2 * k + 1] = std::sin(pi * (double)k / N);
        }
        if (cudaMemcpy(d, t.data(), t.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
            return QG_ERR_CUDA;
    } else {
        std::vector<float> t(2 * n);
        for (size_t k = 0; k < n; ++k) {
            t[2 * k] = (float)std::cos(pi * (double)k / N);
            t[2 * k + 1] = (float)std::sin(pi * (double)k / N);
        }
        if (cudaMemcpy(d, t.data(), t.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return QG_ERR_CUDA;
    }
    h->twcache[N] = d;
    *out = d;
    return QG_OK;
}

qg_status upload_real(qg_ctx* h, void** out, const std::vector<double>& v) {
    qg_status s = dev_alloc(h, out, v.size() * h->esz);
    if (s != QG_OK) return s;
    cudaError_t e;
    if (h->dtype == QG_F64) {
        e = cudaMemcpy(*out, v.data(), v.size() * 8, cudaMemcpyHostToDevice);
    } else {
        std::vector<float> f(v.begin(), v.end());
        e = cudaMemcpy(*out, f.data(), f.size() * 4, cudaMemcpyHostToDevice);
    }
    return e == cudaSuccess ? QG_OK : QG_ERR_CUDA;
}

// Per-pass twiddles of the radix-32 engine for FFT length L (cached).
qg_status get_pass_table(qg_ctx* h, int L, int rad, void** out) {
    const int key = -(L * 64 + rad);   // shares the twiddle cache; negative keys
    auto it = h->twcache.find(key);
    if (it != h->twcache.end()) {
        *out = it->second;
        return QG_OK;
    }
    const size_t n = pass_table_size(L, rad);
    std::vector<double> re(n + 1), im(n + 1), v(2 * (n + 1));
    pass_table(L, rad, re.data(), im.data());
    for (size_t k = 0; k <= n; ++k) {
        v[2 * k] = re[k];
        v[2 * k + 1] = im[k];
    }
    void* d = nullptr;
    qg_status s = upload_real(h, &d, v);
    if (s != QG_OK) return s;
    h->twcache[key] = d;
    *out = d;
    return QG_OK;
}

// Eigenvalue and twiddle tables of grid level `lv` (Eq. ialpha without Ro).
qg_status get_level(qg_ctx* h, int lv, const LevelTables** out) {
    auto it = h->tables.find(lv);
    if (it != h->tables.end()) {
        *out = &it->second;
        return QG_OK;
    }
    LevelTables t;
    t.mx = h->nx >> lv;
    t.my = h->ny >> lv;
    if (solve_smem_bytes(t.mx, t.my, h->esz, 4) > 200 * 1024 &&
        solve_smem_bytes(t.mx, t.my, h->esz, 16) > 200 * 1024)
        return QG_ERR_SHAPE;
    t.ldc = padded_ld(t.mx);
    t.dxc = h->dx * (double)(1 << lv);
    t.dyc = h->dy * (double)(1 << lv);
    qg_status s = get_twiddles(h, t.mx, &t.twx);
    if (s == QG_OK) s = get_twiddles(h, t.my, &t.twy);
    for (int r = 0; r < 3 && s == QG_OK; ++r) {
        const int rad = warp_engine_radix(32 + r);
        // radix 16 (r = 1) also serves engine 50
        if (!solve32_supports(t.mx, t.my, rad, h->esz) &&
            !(rad == 16 && stream_supports(t.mx, t.my, h->esz)))
            continue;
        s = get_pass_table(h, 2 * t.mx, rad, &t.ptx[r]);
        if (s == QG_OK) s = get_pass_table(h, 2 * t.my, rad, &t.pty[r]);
    }
    if (s == QG_OK && h->esz == 4 && mtx_supports(t.mx, t.my, 4, h->layers)) {
        std::vector<float> m(mtx_table_floats(t.mx, t.my));
        mtx_table(t.mx, t.my, t.dxc, t.dyc, m.data());
        s = dev_alloc(h, &t.mtab, m.size() * sizeof(float));
        if (s == QG_OK &&
            cudaMemcpy(t.mtab, m.data(), m.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            s = QG_ERR_CUDA;
    }
    if (s == QG_OK && tc_supports(t.mx, t.my, h->esz, h->layers)) {
        std::vector<float> m(tc_table_floats(t.mx, t.my));
        tc_table(t.mx, t.my, t.dxc, t.dyc, m.data());
        s = dev_alloc(h, &t.tctab, m.size() * sizeof(float));
        if (s == QG_OK &&
            cudaMemcpy(t.tctab, m.data(), m.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            s = QG_ERR_CUDA;
    }
    if (s != QG_OK) return s;
    const double pi = 3.14159265358979323846;
    // padded to a multiple of 4 entries: the solve copies them in 16-byte units
    std::vector<double> lx((t.mx + 1 + 3) / 4 * 4, 0.0), ly((t.my + 1 + 3) / 4 * 4, 0.0);
    for (int k = 1; k < t.mx; ++k) lx[k] = (2.0 * std::cos(pi * k / t.mx) - 2.0) / (t.dxc * t.dxc);
    for (int l = 1; l < t.my; ++l) ly[l] = (2.0 * std::cos(pi * l / t.my) - 2.0) / (t.dyc * t.dyc);
    s = upload_real(h, &t.lamx, lx);
    if (s == QG_OK) s = upload_real(h, &t.lamy, ly);
    if (s != QG_OK) return s;
    h->tables[lv] = t;
    *out = &h->tables[lv];
    return QG_OK;
}

// Bench instrumentation: when h->timing is set, each launch of the step is
// bracketed by two externally visible events captured into the graph.
struct KTimer {
    qg_ctx* h;
    cudaStream_t s;
    int cls;
    cudaEvent_t e1 = nullptr, e2 = nullptr;
    KTimer(qg_ctx* h_, cudaStream_t s_, int c) : h(h_), s(s_), cls(c) {
        if (!h->capturing) return;
        h->kernels_per_step += (c == QG_K_SOLVE && h->split_solve) ? 3 : 1;
        if (!h->timing || !(h->timing_mask & (1u << c))) return;
        if (h->ev_next + 2 > h->ev_pool.size()) {
            for (int k = 0; k < 2; ++k) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) return;
                h->ev_pool.push_back(e);
            }
        }
        e1 = h->ev_pool[h->ev_next++];
        e2 = h->ev_pool[h->ev_next++];
        cudaEventRecordWithFlags(e1, s, cudaEventRecordExternal);
    }
    ~KTimer() {
        if (!e1) return;
        cudaEventRecordWithFlags(e2, s, cudaEventRecordExternal);
        h->ev_used.push_back({cls, {e1, e2}});
    }
};

template <typename T>
T* plane(void* base, size_t plane_elems, int layer) {
    return static_cast<T*>(base) + (size_t)layer * plane_elems;
}

// Elliptic solve on one level (one cooperative launch): `in` holds
// `nparts` planes per layer (the restriction's partial sums when 4), tr is
// the transposed scratch (pitch ld_tr, plane pl_tr), work the y-pass output;
// in, work and out have the level's padded layout and plane size pl.  work
// and out may alias; in may alias either.
int engine_rule(int mx, int my);
int engine_for(qg_ctx* h, int mx, int my);

// ---- multigrid (qg_set_solver) -------------------------------------------
// Grids whose sides are within a factor 4 of each other (halving down to a
// shorter side of 2 intervals leaves a line of at most 7 unknowns) and
// whose spacings are within a factor 2 (point Gauss-Seidel with full
// coarsening smooths poorly on strongly anisotropic grids).
bool mg_supports(int mx, int my, double dx, double dy) {
    const int lo = mx < my ? mx : my, hi = mx < my ? my : mx;
    const double r = dx > dy ? dx / dy : dy / dx;
    return lo >= 2 && hi <= 4 * lo && r <= 2.0 + 1e-12;
}

qg_status get_mg(qg_ctx* h, int mx, int my, const MGPlan** out) {
    const long key = (long)mx * 65536 + my;
    auto it = h->mg.find(key);
    if (it != h->mg.end()) {
        *out = &it->second;
        return QG_OK;
    }
    MGPlan p;
    for (int x = mx, y = my;; x /= 2, y /= 2) {
        p.mx.push_back(x);
        p.my.push_back(y);
        p.ld.push_back(padded_ld(x));
        if ((x < y ? x : y) <= 2) break;
    }
    p.nl = (int)p.mx.size();
    // the tail: the longest run of coarsest grids that fits one CTA's shared
    // memory (at least the coarsest grid itself)
    p.tail = p.nl - 1;
    while (p.tail > 0 && p.nl - p.tail < kMaxTail &&
           mg_tail_smem(&p.mx[p.tail - 1], &p.my[p.tail - 1], p.nl - p.tail + 1, h->esz) <=
               160 * 1024)
        --p.tail;
    if (mg_reserve_tail_smem(mg_tail_smem(&p.mx[p.tail], &p.my[p.tail], p.nl - p.tail, h->esz),
                             h->esz) != cudaSuccess)
        return QG_ERR_CUDA;
    p.psi.assign(p.nl, nullptr);
    p.rhs.assign(p.nl, nullptr);
    for (int k = 0; k < p.nl; ++k) {
        const size_t bytes = (size_t)(p.my[k] + 1) * p.ld[k] * h->esz;
        qg_status s = dev_alloc(h, &p.rhs[k], bytes);
        if (s == QG_OK && k > 0) s = dev_alloc(h, &p.psi[k], bytes);
        if (s != QG_OK) return s;
    }
    auto r = h->mg.emplace(key, std::move(p));
    *out = &r.first->second;
    return QG_OK;
}

// lap_h psi = (sum of the nparts planes of `in`) on the grid of t, in place
// in `out` (the guess: out's contents, or zero), with h->mg_cycles V-cycles.
template <typename T>
qg_status mg_solve_level(qg_ctx* h, const LevelTables& t, const void* in, int nparts, void* out,
                         size_t pl, cudaStream_t s, bool zero) {
    const MGPlan* mp = nullptr;
    qg_status st = get_mg(h, t.mx, t.my, &mp);
    if (st != QG_OK) return fail(h, st);
    if (mp->ld[0] != t.ldc) return fail(h, QG_ERR_CUDA);
    MGSumParams<T> q = {};
    for (int k = 0; k < nparts; ++k) q.in[k] = plane<T>(const_cast<void*>(in), pl, k);
    q.nin = nparts;
    q.ld_in = t.ldc;
    q.rhs = static_cast<T*>(mp->rhs[0]);
    q.psi = static_cast<T*>(out);
    q.mx = t.mx;
    q.my = t.my;
    q.ld = t.ldc;
    q.zero = zero ? 1 : 0;
    std::vector<MGLevelDesc<T>> lv(mp->nl);
    double dx = t.dxc, dy = t.dyc;
    for (int k = 0; k < mp->nl; ++k, dx *= 2, dy *= 2) {
        lv[k].psi = k == 0 ? static_cast<T*>(out) : static_cast<T*>(mp->psi[k]);
        lv[k].rhs_w = static_cast<T*>(mp->rhs[k]);
        lv[k].rhs = lv[k].rhs_w;
        lv[k].mx = mp->mx[k];
        lv[k].my = mp->my[k];
        lv[k].ld = lv[k].ldr = mp->ld[k];
        lv[k].cx = (T)(1.0 / (dx * dx));
        lv[k].cy = (T)(1.0 / (dy * dy));
    }
    KTimer kt(h, s, QG_K_SOLVE);
    if (h->capturing) h->kernels_per_step += h->mg_cycles * mg_cycle_launches(mp->tail);
    QG_TRY(launch_mg_sum<T>(q, s));
    for (int c = 0; c < h->mg_cycles; ++c) QG_TRY(launch_mg_cycle<T>(lv.data(), mp->nl, mp->tail, s));
    return QG_OK;
}

template <typename T>
qg_status solve_level(qg_ctx* h, const LevelTables& t, const void* in, void* tr, int ld_tr,
                      size_t pl_tr, void* work, void* out, size_t pl, cudaStream_t s,
                      int nparts = 1, int engine = 0) {
    using C = typename Cx<T>::type;
    if (h->solver == QG_SOLVER_MULTIGRID && h->layers == 1)
        return mg_solve_level<T>(h, t, in, nparts, out, pl, s, false);
    SolveParams<T> P = {};
    P.mx = t.mx;
    P.my = t.my;
    P.layers = h->layers;
    for (int L = 0; L < h->layers; ++L) {
        for (int q = 0; q < nparts; ++q)
            P.in[L][q] = plane<T>(const_cast<void*>(in), pl, L * nparts + q);
        P.tr[L] = plane<T>(tr, pl_tr, L);
        P.work[L] = plane<T>(work, pl, L);
        P.out[L] = plane<T>(out, pl, L);
    }
    P.nin = nparts;
    P.part_px = P.part_py = 1;
    if (nparts > 1) {
        P.part_px = fine_part_period_x(h->levels);
        P.part_py = fine_part_period_y(h->levels, h->fine_rows);
    }
    P.ld = t.ldc;
    P.ld_tr = ld_tr;
    P.twx = static_cast<const C*>(t.twx);
    P.twy = static_cast<const C*>(t.twy);
    const int eng = engine ? engine : engine_for(h, t.mx, t.my);
    const int tab = eng == kStreamEngine ? 1 : eng - 32;   // engine 50: radix-16 tables
    const bool fft_tab = is_warp_engine(eng) || eng == kStreamEngine;
    P.ptx = fft_tab ? static_cast<const C*>(t.ptx[tab]) : nullptr;
    P.pty = fft_tab ? static_cast<const C*>(t.pty[tab]) : nullptr;
    P.lamx = static_cast<const T*>(t.lamx);
    P.lamy = static_cast<const T*>(t.lamy);
    P.scale = (T)((2.0 / t.mx) * (2.0 / t.my));
    P.Ro = (T)h->Ro;
    if (h->layers == 2) {
        P.f1 = (T)(h->Fr / h->delta);
        P.f2 = (T)(h->Fr / (1.0 - h->delta));
    }
    P.bar = h->dbar;
    P.bar_extra = h->fault == QG_FAULT_BARRIER_STALL ? 1u : 0u;
    P.err = h->derr;
    P.split = h->split_solve ? 1 : 0;
    KTimer kt(h, s, QG_K_SOLVE);
    if (h->capturing && !h->split_solve) h->kernels_per_step += solve_launches(eng) - 1;
    if (eng == kMatrixEngine || eng == kTcEngine) {
        // one launch whether or not the FFT solves are split
        if (h->capturing && h->split_solve) h->kernels_per_step -= 2;
        if constexpr (std::is_same<T, float>::value) {
            QG_TRY(eng == kTcEngine
                       ? launch_solve_tc(P, static_cast<const float*>(t.tctab), s)
                       : launch_solve_mtx(P, static_cast<const float*>(t.mtab), s));
        } else {
            QG_TRY(cudaErrorInvalidValue);
        }
        return QG_OK;
    }
    QG_TRY(launch_solve<T>(P, eng, s));
    return QG_OK;
}

// ---- solve-engine autotuner ---------------------------------------------
// The FFT engine of the solve (shared-memory Stockham engine with base
// radix 4: many threads per sequence pair, or 16: fewer passes and
// instructions; or the warp-group engine of solve32.cu with 32, 16 or 8
// values per thread, engines 32, 33, 34; or, on small one-layer FP32 grids,
// the matrix-form solve on the tensor cores of solve_mtx.cu, engine 40, or
// the same with tcgen05 and TMEM accumulators, engine 41 (solve_tc.cu); or
// the register-resident radix-16 passes of solve_stream.cu, engine 50) is
// chosen per handle when it is created, by timing a few whole steps with each
// engine that supports the elliptic grid (the solve alone, timed back to
// back, ranks them differently: in a step the fine sweep has just streamed
// its fields through L2), and the fastest is kept.  Results are cached per
// (nx, ny, levels, layers, dtype) for the process and, when the environment
// variable QG_TUNE_CACHE names a file, in that file (one line
// "nx ny levels layers esz engine rows ry" per entry; ensemble groups add
// lines "group mx my dx dy members esz engine").  QG_SOLVE_ENGINE=4|16|32|33|34|40|41|50
// forces a choice where that engine supports the grid.  Other grids use the
// size rule.

int engine_rule(int mx, int my) { return (long)mx * my >= (1L << 21) ? 16 : 4; }

int engine_for(qg_ctx* h, int mx, int my) {
    const LevelTables* t = nullptr;
    if (get_level(h, h->levels, &t) == QG_OK && t->mx == mx && t->my == my) return h->solve_engine;
    return engine_rule(mx, my);
}

// Whether engine e can solve the level with tables t on handle h.
bool engine_ok(const qg_ctx* h, const LevelTables* t, size_t esz, int e) {
    if (e == kMatrixEngine) return t->mtab && mtx_supports(t->mx, t->my, esz, h->layers);
    if (e == kTcEngine) return t->tctab && tc_supports(t->mx, t->my, esz, h->layers);
    if (e == kStreamEngine) return solve_engine_supports(t->mx, t->my, esz, e) && t->ptx[1];
    return solve_engine_supports(t->mx, t->my, esz, e) && (!is_warp_engine(e) || t->ptx[e - 32]);
}

// TMA tensor maps of the fine buffers for the handle's tile height: halo
// boxes of w^(s) and the fine psi, interior boxes of w^n and the forcing.
qg_status fine_maps(qg_ctx* h) {
    const int rows = h->fine_rows;
    for (int k = 0; k < 3; ++k) {
        for (int L = 0; L < h->layers; ++L) {
            const void* base = static_cast<const char*>(h->w[k]) + L * h->plane_f * h->esz;
            if (make_tensor_map(&h->tm_halo[k][L], base, h->nx, h->ny, h->ldf, h->esz,
                                fine_halo_cols(), rows + 2) != cudaSuccess ||
                make_tensor_map(&h->tm_int[k][L], base, h->nx, h->ny, h->ldf, h->esz,
                                fine_block_cols(), rows) != cudaSuccess)
                return QG_ERR_CUDA;
        }
    }
    if (make_tensor_map(&h->tm_psi, h->psi, h->nx, h->ny, h->ldf, h->esz, fine_halo_cols(),
                        rows + 2) != cudaSuccess)
        return QG_ERR_CUDA;
    if (h->f2d) {
        if (make_tensor_map(&h->tm_f, h->f2d, h->nx, h->ny, h->ldf, h->esz, fine_block_cols(),
                            rows) != cudaSuccess)
            return QG_ERR_CUDA;
    } else {
        h->tm_f = h->tm_int[0][0];
    }
    return QG_OK;
}

using TuneKey = std::tuple<int, int, int, int, int>;
std::mutex g_tune_mutex;
struct TuneVal {
    int engine, rows, ry;   // solve engine; fine rows per CTA and per thread
};
std::map<TuneKey, TuneVal> g_tune_cache;
bool g_tune_file_read = false;
// ensemble groups' solve engines by (elliptic grid, spacings, members, dtype)
using GroupKey = std::tuple<int, int, double, double, int, int>;
std::mutex g_batch_tune_mutex;
std::map<GroupKey, int> g_batch_tune;

bool known_engine(int e) {
    return e == 4 || e == 16 || is_warp_engine(e) || e == kMatrixEngine || e == kTcEngine ||
           e == kStreamEngine;
}

// (called with g_tune_mutex held)
void tune_file_load() {
    if (g_tune_file_read) return;
    g_tune_file_read = true;
    const char* path = std::getenv("QG_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[256];
    while (std::fgets(line, sizeof line, f)) {
        int a, b, c, d, x, e, r, y;
        double dx, dy;
        if (std::sscanf(line, "group %d %d %lf %lf %d %d %d", &a, &b, &dx, &dy, &c, &x, &e) == 7) {
            if (known_engine(e)) {
                std::lock_guard<std::mutex> lock(g_batch_tune_mutex);
                g_batch_tune[GroupKey(a, b, dx, dy, c, x)] = e;
            }
        } else if (std::sscanf(line, "%d %d %d %d %d %d %d %d", &a, &b, &c, &d, &x, &e, &r, &y) == 8 &&
                   known_engine(e) && fine_rows_supported((size_t)x, d, c, r, y)) {
            g_tune_cache[TuneKey(a, b, c, d, x)] = {e, r, y};
        }
    }
    std::fclose(f);
}

void tune_file_store(const TuneKey& k, const TuneVal& v) {
    const char* path = std::getenv("QG_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%d %d %d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k),
                 std::get<3>(k), std::get<4>(k), v.engine, v.rows, v.ry);
    std::fclose(f);
}

void tune_file_store_group(const GroupKey& k, int engine) {
    const char* path = std::getenv("QG_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "group %d %d %.17g %.17g %d %d %d\n", std::get<0>(k), std::get<1>(k),
                 std::get<2>(k), std::get<3>(k), std::get<4>(k), std::get<5>(k), engine);
    std::fclose(f);
}

qg_status build_graph(qg_ctx* h);
void drop_graph(qg_ctx* h);
template <typename T>
qg_status init_partials(qg_ctx* h, cudaStream_t s);

// Milliseconds of 5 captured steps with solve engine `engine` (after 3
// untimed ones), run on the handle's own buffers.
template <typename T>
float time_steps(qg_ctx* h, int engine) {
    const LevelTables* t = nullptr;
    if (get_level(h, h->levels, &t) != QG_OK) return 1e30f;
    if (!engine_ok(h, t, sizeof(T), engine)) return 1e30f;
    h->solve_engine = engine;
    drop_graph(h);
    if (build_graph(h) != QG_OK) return 1e30f;
    if (h->part && init_partials<T>(h, h->stream) != QG_OK) return 1e30f;
    for (int k = 0; k < 3; ++k)
        if (cudaGraphLaunch(h->gexec, h->stream) != cudaSuccess) return 1e30f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return 1e30f;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return 1e30f;
    }
    float ms = 1e30f;
    bool ok = cudaEventRecord(e0, h->stream) == cudaSuccess;
    for (int k = 0; k < 5 && ok; ++k) ok = cudaGraphLaunch(h->gexec, h->stream) == cudaSuccess;
    ok = ok && cudaEventRecord(e1, h->stream) == cudaSuccess;
    if (ok && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

// Zero the state, streamfunction and scratch arrays of a handle whose
// buffers ran timing steps (autotuners), and wait for it.
qg_status rest_buffers(qg_ctx* h, cudaStream_t s) {
    cudaStreamSynchronize(s);
    for (void* p : {h->w[0], h->w[1], h->w[2], h->psi}) {
        if (p) QG_TRY(cudaMemsetAsync(p, 0, h->plane_f * h->layers * h->esz, s));
    }
    for (void* p : {h->cw, h->cpsi}) {
        if (p) QG_TRY(cudaMemsetAsync(p, 0, h->plane_c * h->layers * h->esz, s));
    }
    if (h->ct) QG_TRY(cudaMemsetAsync(h->ct, 0, h->plane_t * h->layers * h->esz, s));
    if (h->part)
        QG_TRY(cudaMemsetAsync(h->part, 0, 4 * (size_t)h->layers * h->plane_c * h->esz, s));
    QG_TRY(cudaMemsetAsync(h->dclock, 0, sizeof(double) * 4, s));
    h->part_valid = false;
    QG_TRY(cudaStreamSynchronize(s));
    return QG_OK;
}

template <typename T>
qg_status autotune_solve(qg_ctx* h) {
    const LevelTables* t = nullptr;
    qg_status st = get_level(h, h->levels, &t);
    if (st != QG_OK) return st;
    // the tiles the fused fine stage may take on this handle: (rows per CTA,
    // rows per thread); ensemble members keep the default (their batched
    // sweep uses it)
    using Tile = std::pair<int, int>;
    std::vector<Tile> tiles{{h->fine_rows, h->fine_ry}};
    if (!h->member)
        for (Tile c : {Tile{64, h->fine_ry}, Tile{32, h->fine_ry}, Tile{64, 4}, Tile{32, 4}})
            if (c != tiles[0] && fine_rows_supported(h->esz, h->layers, h->levels, c.first, c.second))
                tiles.push_back(c);
    // QG_FINE_ROWS=<rows> or <rows>x<rows per thread> forces an offered tile
    Tile forced{0, 0};
    if (const char* fr = std::getenv("QG_FINE_ROWS")) {
        int r = 0, y = 0;
        const int n = std::sscanf(fr, "%dx%d", &r, &y);
        if (n == 1) y = fine_rows_per_thread(h->levels);
        const Tile c{r, y};
        if (n >= 1 && std::find(tiles.begin(), tiles.end(), c) != tiles.end()) forced = c;
    }
    auto set_tile = [&](Tile c) -> qg_status {
        if (c.first == h->fine_rows && c.second == h->fine_ry) return QG_OK;
        h->fine_rows = c.first;
        h->fine_ry = c.second;
        drop_graph(h);
        return fine_maps(h);
    };
    const bool forced_rows = forced.first != 0;
    if (forced_rows) QG_TRY_S(set_tile(forced));
    if (const char* force = std::getenv("QG_SOLVE_ENGINE")) {
        const int e = std::atoi(force);
        if (engine_ok(h, t, sizeof(T), e)) {
            h->solve_engine = e;
            h->engine_forced = true;
            return QG_OK;
        }
    }
    const TuneKey key(h->nx, h->ny, h->levels, h->layers, (int)h->esz);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        tune_file_load();
        auto it = g_tune_cache.find(key);
        const Tile cached{it == g_tune_cache.end() ? 0 : it->second.rows,
                          it == g_tune_cache.end() ? 0 : it->second.ry};
        if (it != g_tune_cache.end() &&
            std::find(tiles.begin(), tiles.end(), cached) != tiles.end()) {
            h->solve_engine = it->second.engine;
            if (!forced_rows) QG_TRY_S(set_tile(cached));
            return QG_OK;
        }
    }
    const float t4 = time_steps<T>(h, 4);
    const float t32 = time_steps<T>(h, 32);
    const float t33 = time_steps<T>(h, 33);
    const float t34 = time_steps<T>(h, 34);
    const float t16 = time_steps<T>(h, 16);
    const float t40 = time_steps<T>(h, kMatrixEngine);
    const float t50 = time_steps<T>(h, kStreamEngine);
    const float t41 = time_steps<T>(h, kTcEngine);
    // a candidate that cannot run on this grid is a tuning result, not an error
    h->latched = QG_OK;
    (void)cudaGetLastError();
    drop_graph(h);
    const float tt[8] = {t4, t16, t32, t33, t34, t40, t50, t41};
    const int ee[8] = {4, 16, 32, 33, 34, kMatrixEngine, kStreamEngine, kTcEngine};
    int best = 0;
    for (int k = 1; k < 8; ++k)
        if (tt[k] < tt[best]) best = k;
    if (tt[best] >= 1e29f) return fail(h, QG_ERR_CUDA);
    h->solve_engine = ee[best];
    // then the fine stage's tile, with that engine
    if (!forced_rows && tiles.size() > 1) {
        float tbest = tt[best];
        Tile cbest = tiles[0];
        for (size_t k = 1; k < tiles.size(); ++k) {
            if (set_tile(tiles[k]) != QG_OK) break;
            const float tr = time_steps<T>(h, h->solve_engine);
            if (tr < tbest) {
                tbest = tr;
                cbest = tiles[k];
            }
        }
        h->latched = QG_OK;
        (void)cudaGetLastError();
        QG_TRY_S(set_tile(cbest));
        drop_graph(h);
    }
    // the timing steps ran on the handle's buffers: return them to rest
    QG_TRY_S(rest_buffers(h, h->stream));
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    const TuneVal v{h->solve_engine, h->fine_rows, h->fine_ry};
    g_tune_cache[key] = v;
    tune_file_store(key, v);
    return QG_OK;
}

// CGP steps (ii)-(iv): fine state planes -> fine psi planes (into `out`).
template <typename T>
qg_status project_to(qg_ctx* h, const void* win, void* out, cudaStream_t s) {
    const LevelTables* t = nullptr;
    qg_status st = get_level(h, h->levels, &t);
    if (st != QG_OK) return fail(h, st);
    if (h->levels == 0) {
        return solve_level<T>(h, *t, win, h->ct, h->ld_t, h->plane_t, h->cw, out,
                              h->plane_f, s);
    }
    for (int L = 0; L < h->layers; ++L) {
        KTimer kt(h, s, QG_K_RESTRICT);
        QG_TRY(launch_restrict<T>(plane<T>(const_cast<void*>(win), h->plane_f, L), h->ldf,
                                  plane<T>(h->cw, h->plane_c, L), t->ldc, t->mx, t->my,
                                  h->levels, s));
    }
    st = solve_level<T>(h, *t, h->cw, h->ct, h->ld_t, h->plane_t, h->cw, h->cpsi,
                        h->plane_c, s);
    if (st != QG_OK) return st;
    for (int L = 0; L < h->layers; ++L) {
        KTimer kt(h, s, QG_K_PROLONG);
        QG_TRY(launch_prolong<T>(plane<T>(h->cpsi, h->plane_c, L), t->ldc,
                                 plane<T>(out, h->plane_f, L), h->ldf, h->nx, h->ny,
                                 h->levels, s));
    }
    return QG_OK;
}

template <typename T>
qg_status project(qg_ctx* h, const void* win, cudaStream_t s) {
    return project_to<T>(h, win, h->psi, s);
}

// TVDRK3 stage s: w_out = a w^n + b (w_in + dt G(w_in)).
template <typename T>
qg_status stage(qg_ctx* h, int s_idx, cudaStream_t s) {
    static const double A[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double B[3] = {1.0, 0.25, 2.0 / 3.0};
    void* win = h->w[s_idx];
    void* wout = h->w[(s_idx + 1) % 3];
    qg_status st = project<T>(h, win, s);
    if (st != QG_OK) return st;
    if (h->stats && s_idx == 0) {
        QG_TRY(launch_accumulate<T>(h->stat_acc, static_cast<const T*>(h->psi),
                                    h->plane_f * h->layers, s));
        QG_TRY(launch_accumulate<T>(h->stat_acc_w, static_cast<const T*>(h->w[0]),
                                    h->plane_f * h->layers, s));
    }
    KTimer kt(h, s, QG_K_FINE);
    if (h->layers == 1) {
        StageParams<T> p;
        p.nx = h->nx;
        p.ny = h->ny;
        p.ld = h->ldf;
        p.c_jac = (T)(1.0 / (12.0 * h->dx * h->dy));
        p.c_beta = (T)(1.0 / (12.0 * h->Ro * h->dx));
        p.c_lapx = (T)(1.0 / (h->Re * h->dx * h->dx));
        p.c_lapy = (T)(1.0 / (h->Re * h->dy * h->dy));
        p.dt = (T)h->dt;
        p.a = (T)A[s_idx];
        p.b = (T)B[s_idx];
        QG_TRY(launch_fine_stage<T>(static_cast<const T*>(h->psi),
                                    static_cast<const T*>(win),
                                    static_cast<const T*>(h->w[0]),
                                    static_cast<T*>(wout),
                                    static_cast<const T*>(h->frow),
                                    static_cast<const T*>(h->f2d), p, s));
    } else {
        StageParams2<T> p;
        p.nx = h->nx;
        p.ny = h->ny;
        p.ld = h->ldf;
        p.c_jac = (T)(1.0 / (12.0 * h->dx * h->dy));
        p.c_beta = (T)(1.0 / (12.0 * h->dx));
        p.inv_Ro = (T)(1.0 / h->Ro);
        p.f1 = (T)(h->Fr / h->delta);
        p.f2 = (T)(h->Fr / (1.0 - h->delta));
        const double A2 = h->Ro / h->Re;
        p.A_dx2 = (T)(A2 / (h->dx * h->dx));
        p.A_dy2 = (T)(A2 / (h->dy * h->dy));
        p.sigma = (T)h->sigma;
        p.dt = (T)h->dt;
        p.a = (T)A[s_idx];
        p.b = (T)B[s_idx];
        const size_t P = h->plane_f;
        QG_TRY(launch_fine_stage2<T>(plane<T>(h->psi, P, 0), plane<T>(h->psi, P, 1),
                                     plane<T>(win, P, 0), plane<T>(win, P, 1),
                                     plane<T>(h->w[0], P, 0), plane<T>(h->w[0], P, 1),
                                     plane<T>(wout, P, 0), plane<T>(wout, P, 1),
                                     static_cast<const T*>(h->frow), p, s));
    }
    return QG_OK;
}

// Two-layer stage with the fused fine kernel (l >= 1): the coupled solve of
// both layers from their partial planes has run; one fused launch per layer
// prolongs both psi (its own for the Jacobian and the beta term, both for
// the relative vorticity of the dissipation, Eq. pv-non), updates Q_i and
// leaves R^l Q_i^(s+1) in that layer's partial planes.
template <typename T>
qg_status stage_fused2(qg_ctx* h, int s_idx, const LevelTables& t, cudaStream_t s) {
    static const double A[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double B[3] = {1.0, 0.25, 2.0 / 3.0};
    void* win = h->w[s_idx];
    void* wout = h->w[(s_idx + 1) % 3];
    const double Av = h->Ro / h->Re;    // lateral eddy viscosity A (Re = Ro/A)
    // The layers' fine stages are independent (each reads both layers' psi
    // and writes only its own fields and partial planes): the second runs on
    // a branch beside the first, so that the two half-GPU grids fill it.
    cudaStream_t s1 = h->side ? h->side : s;
    if (s1 != s) {
        QG_TRY(cudaEventRecord(h->ev_fork, s));
        QG_TRY(cudaStreamWaitEvent(s1, h->ev_fork, 0));
    }
    for (int L = 0; L < 2; ++L) {
        const cudaStream_t sl = L == 1 ? s1 : s;
        FusedParams<T> p;
        p.nx = h->nx;
        p.ny = h->ny;
        p.ld = h->ldf;
        p.psi = plane<T>(h->cpsi, h->plane_c, L);
        p.psi_o = plane<T>(h->cpsi, h->plane_c, 1 - L);
        p.ldp = t.ldc;
        p.w = plane<T>(win, h->plane_f, L);
        p.wn = plane<T>(h->w[0], h->plane_f, L);
        p.wout = plane<T>(wout, h->plane_f, L);
        p.frow = L == 0 ? static_cast<const T*>(h->frow) : nullptr;
        p.f2d = nullptr;
        for (int q = 0; q < 4; ++q) p.part[q] = plane<T>(h->part, h->plane_c, 4 * L + q);
        p.ldc = t.ldc;
        p.err = h->derr;
        p.c_jac = (T)(1.0 / (12.0 * h->dx * h->dy));
        p.c_beta = (T)(1.0 / (12.0 * h->dx));
        p.c_lapx = (T)(Av / (h->dx * h->dx));
        p.c_lapy = (T)(Av / (h->dy * h->dy));
        p.dt = (T)h->dt;
        p.a = (T)A[s_idx];
        p.b = (T)B[s_idx];
        p.inv_Ro = (T)(1.0 / h->Ro);
        p.k_p = (T)((L == 0 ? h->Fr / h->delta : h->Fr / (1.0 - h->delta)) / h->Ro);
        p.drag = L == 1 ? (T)h->sigma : T(0);
        p.umax = nullptr;
        p.cfl_h = 0.0;
        p.dt_cap = h->dt;
        p.clock = h->dclock + 1;
        p.last_stage = s_idx == 2 && L == 1;
        FineMaps m;
        m.w = h->tm_halo[s_idx][L];
        m.wn = h->tm_int[0][L];
        m.psi = h->tm_psi;
        m.f = h->tm_f;
        KTimer kt(h, sl, QG_K_FINE);
        QG_TRY(launch_fine_fused<T>(p, m, h->levels, sl, true, h->fine_rows, h->fine_ry));
    }
    if (s1 != s) {
        QG_TRY(cudaEventRecord(h->ev_join, s1));
        QG_TRY(cudaStreamWaitEvent(s, h->ev_join, 0));
    }
    return QG_OK;
}

// One-layer stage with the fused fine kernel.  On entry the restriction of
// w^(s) is in the partial planes (l >= 1) or w^(s) itself is the elliptic
// right-hand side (l = 0); the stage solves for psibar^(s), then the fused
// kernel prolongs it, updates the fine state and leaves R^l w^(s+1) in the
// partial planes for the next stage.
template <typename T>
qg_status stage_fused(qg_ctx* h, int s_idx, cudaStream_t s) {
    static const double A[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double B[3] = {1.0, 0.25, 2.0 / 3.0};
    void* win = h->w[s_idx];
    void* wout = h->w[(s_idx + 1) % 3];
    const LevelTables* t = nullptr;
    qg_status st = get_level(h, h->levels, &t);
    if (st != QG_OK) return fail(h, st);
    if (h->levels == 0) {
        st = solve_level<T>(h, *t, win, h->ct, h->ld_t, h->plane_t, h->cw, h->psi,
                            h->plane_f, s, 1);
    } else {
        st = solve_level<T>(h, *t, h->part, h->ct, h->ld_t, h->plane_t, h->cw, h->cpsi,
                            h->plane_c, s, 4);
    }
    if (st != QG_OK) return st;
    if (h->stats && s_idx == 0) {
        const bool fine = h->levels == 0;
        QG_TRY(launch_accumulate<T>(h->stat_acc, static_cast<const T*>(fine ? h->psi : h->cpsi),
                                    (fine ? h->plane_f : h->plane_c) * h->layers, s));
        QG_TRY(launch_accumulate<T>(h->stat_acc_w, static_cast<const T*>(h->w[0]),
                                    h->plane_f * h->layers, s));
    }
    if (h->layers == 2) return stage_fused2<T>(h, s_idx, *t, s);
    FusedParams<T> p;
    p.nx = h->nx;
    p.ny = h->ny;
    p.ld = h->ldf;
    p.psi = static_cast<const T*>(h->levels == 0 ? h->psi : h->cpsi);
    p.ldp = h->levels == 0 ? h->ldf : t->ldc;
    p.w = static_cast<const T*>(win);
    p.wn = static_cast<const T*>(h->w[0]);
    p.wout = static_cast<T*>(wout);
    p.frow = static_cast<const T*>(h->frow);
    p.f2d = static_cast<const T*>(h->f2d);
    for (int q = 0; q < 4; ++q)
        p.part[q] = h->part ? plane<T>(h->part, h->plane_c, q) : nullptr;
    p.ldc = t->ldc;
    p.err = h->derr;
    p.c_jac = (T)(1.0 / (12.0 * h->dx * h->dy));
    p.c_beta = (T)(1.0 / (12.0 * h->Ro * h->dx));
    p.c_lapx = (T)(1.0 / (h->Re * h->dx * h->dx));
    p.c_lapy = (T)(1.0 / (h->Re * h->dy * h->dy));
    p.dt = (T)h->dt;
    p.a = (T)A[s_idx];
    p.b = (T)B[s_idx];
    p.psi_o = nullptr;
    p.inv_Ro = p.k_p = p.drag = T(0);
    p.umax = nullptr;
    p.cfl_h = h->cfl * std::fmin(h->dx, h->dy);
    p.dt_cap = h->dt;
    p.clock = h->dclock + 1;
    p.last_stage = s_idx == 2;
    if (h->cfl > 0.0) {
        p.umax = reinterpret_cast<const unsigned long long*>(h->dclock);
        if (s_idx == 0) {
            // Eq. dt from psi^n, the streamfunction of this first stage
            QG_TRY(cudaMemsetAsync(h->dclock, 0, sizeof(double), s));
            KTimer kc(h, s, QG_K_CFL);
            QG_TRY(launch_cfl_max<T>(static_cast<const T*>(p.psi), p.ldp, h->nx, h->ny,
                                     h->levels, h->dx, h->dy,
                                     reinterpret_cast<unsigned long long*>(h->dclock), s));
        }
    }
    FineMaps m;
    m.w = h->tm_halo[s_idx][0];
    m.wn = h->tm_int[0][0];
    m.psi = h->tm_psi;
    m.f = h->tm_f;
    KTimer kt(h, s, QG_K_FINE);
    QG_TRY(launch_fine_fused<T>(p, m, h->levels, s, false, h->fine_rows, h->fine_ry));
    return QG_OK;
}

// Restriction of the current state into the partial planes (plane 0 holds
// the complete values, planes 1-3 zero), needed once after qg_set_state.
template <typename T>
qg_status init_partials(qg_ctx* h, cudaStream_t s) {
    const LevelTables* t = nullptr;
    qg_status st = get_level(h, h->levels, &t);
    if (st != QG_OK) return fail(h, st);
    QG_TRY(cudaMemsetAsync(h->part, 0, 4 * (size_t)h->layers * h->plane_c * sizeof(T), s));
    for (int L = 0; L < h->layers; ++L)
        QG_TRY(launch_restrict<T>(plane<T>(h->w[0], h->plane_f, L), h->ldf,
                                  plane<T>(h->part, h->plane_c, 4 * L), t->ldc, t->mx, t->my,
                                  h->levels, s));
    return QG_OK;
}

template <typename T>
qg_status enqueue_step(qg_ctx* h, cudaStream_t s) {
    for (int k = 0; k < 3; ++k) {
        // the fused path: one layer at any level, two layers when coarsened
        qg_status st = (h->layers == 1 || h->levels >= 1) ? stage_fused<T>(h, k, s)
                                                          : stage<T>(h, k, s);
        if (st != QG_OK) return st;
    }
    return QG_OK;
}

qg_status enqueue_step_any(qg_ctx* h, cudaStream_t s) {
    return h->dtype == QG_F64 ? enqueue_step<double>(h, s) : enqueue_step<float>(h, s);
}

qg_status project_any(qg_ctx* h, const void* win, cudaStream_t s) {
    return h->dtype == QG_F64 ? project<double>(h, win, s) : project<float>(h, win, s);
}

void drop_graph(qg_ctx* h) {
    ++h->graph_gen;
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
}

qg_status build_graph(qg_ctx* h) {
    if (h->gexec) return QG_OK;
    h->ev_next = 0;
    h->ev_used.clear();
    h->kernels_per_step = 0;
    QG_TRY(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    qg_status st = enqueue_step_any(h, h->cap);
    h->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap, &g);
    if (st != QG_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_status(h, e);
    h->graph = g;
    QG_TRY(cudaGraphInstantiate(&h->gexec, g, 0));
    return QG_OK;
}

bool pow2_in(int v, int lo, int hi) { return is_pow2(v) && v >= lo && v <= hi; }

}  // namespace

extern "C" {

const char* qg_status_string(qg_status s) {
    switch (s) {
        case QG_OK: return "ok";
        case QG_ERR_ARG: return "invalid argument";
        case QG_ERR_SHAPE: return "unsupported grid shape";
        case QG_ERR_CUDA: return "CUDA error";
        case QG_ERR_OOM: return "device out of memory";
        case QG_ERR_NONFINITE: return "state is not finite";
        case QG_ERR_CFL: return "Courant number above 1 (Eq. dt)";
        case QG_ERR_TIMEOUT: return "device wait timed out";
        case QG_ERR_UNSUPPORTED: return "unsupported request";
        case QG_ERR_NO_DEVICE: return "no CUDA device";
    }
    return "unknown status";
}

static qg_status create_ctx(const qg_basin* b, int layers, double Re, double Ro, double Fr,
                            int levels, qg_dtype dtype, void* cuda_stream, bool split,
                            qg_handle* out);

qg_status qg_create(const qg_basin* b, int layers, double Re, double Ro, double Fr,
                    int levels, qg_dtype dtype, void* cuda_stream, qg_handle* out) {
    return create_ctx(b, layers, Re, Ro, Fr, levels, dtype, cuda_stream, false, out);
}

static qg_status create_ctx(const qg_basin* b, int layers, double Re, double Ro, double Fr,
                            int levels, qg_dtype dtype, void* cuda_stream, bool split,
                            qg_handle* out) {
    if (!b || !out) return QG_ERR_ARG;
    *out = nullptr;
    if (layers != 1 && layers != 2) return QG_ERR_ARG;
    if (dtype != QG_F32 && dtype != QG_F64) return QG_ERR_ARG;
    if (b->flags != 0) return QG_ERR_ARG;
    if (!(Re > 0) || !(Ro > 0) || !(b->dt > 0) || !(b->x1 > b->x0) || !(b->y1 > b->y0))
        return QG_ERR_ARG;
    if (!std::isfinite(Re) || !std::isfinite(Ro) || !std::isfinite(b->dt)) return QG_ERR_ARG;
    if (layers == 2 && (!(b->delta > 0) || !(b->delta < 1) || !(Fr >= 0) || !(b->sigma >= 0)))
        return QG_ERR_ARG;
    if (levels < 0 || levels > 4) return QG_ERR_ARG;
    if (!pow2_in(b->nx, 8, 8192) || !pow2_in(b->ny, 8, 8192)) return QG_ERR_SHAPE;
    if ((b->nx >> levels) < 8 || (b->ny >> levels) < 8) return QG_ERR_SHAPE;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        (void)cudaGetLastError();
        return QG_ERR_NO_DEVICE;
    }
    qg_ctx* h = new (std::nothrow) qg_ctx();
    if (!h) return QG_ERR_OOM;
    h->layers = layers;
    h->dtype = dtype;
    h->esz = dtype == QG_F64 ? 8 : 4;
    h->nx = b->nx;
    h->ny = b->ny;
    h->levels = levels;
    h->x0 = b->x0; h->x1 = b->x1; h->y0 = b->y0; h->y1 = b->y1;
    h->dx = (b->x1 - b->x0) / b->nx;
    h->dy = (b->y1 - b->y0) / b->ny;
    h->Re = Re; h->Ro = Ro; h->Fr = Fr;
    h->delta = b->delta; h->sigma = b->sigma; h->dt = b->dt; h->amp = b->forcing_amp;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->split_solve = split;
    h->member = split;   // ensemble members are the handles created with split solves
    h->ldf = padded_ld(h->nx);
    h->plane_f = (size_t)(h->ny + 1) * h->ldf;
    const int mx = h->nx >> levels, my = h->ny >> levels;
    h->plane_c = (size_t)(my + 1) * padded_ld(mx);
    qg_status s = QG_OK;
    auto guard = [&](qg_status st) {
        if (st != QG_OK && s == QG_OK) s = st;
    };
    if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) guard(QG_ERR_CUDA);
    if (s == QG_OK && layers == 2 &&
        (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess))
        guard(QG_ERR_CUDA);

    const size_t fb = h->plane_f * layers * h->esz;
    const size_t cb = h->plane_c * layers * h->esz;
    for (int k = 0; k < 3 && s == QG_OK; ++k) guard(dev_alloc(h, &h->w[k], fb));
    if (s == QG_OK) guard(dev_alloc(h, &h->psi, fb));
    if (s == QG_OK) guard(dev_alloc(h, &h->cw, cb));
    if (s == QG_OK) guard(dev_alloc(h, &h->cpsi, cb));
    h->ld_t = padded_ld(my);
    h->plane_t = (size_t)(mx + 1) * h->ld_t;
    if (s == QG_OK) guard(dev_alloc(h, &h->ct, h->plane_t * layers * h->esz));
    if (s == QG_OK && levels >= 1)
        guard(dev_alloc(h, &h->part, 4 * (size_t)layers * h->plane_c * h->esz));
    if (s == QG_OK) guard(dev_alloc(h, (void**)&h->derr, sizeof(int) * 4));
    if (s == QG_OK) guard(dev_alloc(h, (void**)&h->dbar, sizeof(unsigned) * 4));
    if (s == QG_OK) guard(dev_alloc(h, (void**)&h->dclock, sizeof(double) * 4));
    if (s == QG_OK) {
        // ensemble members (one layer) sweep the tile of the batched launch
        h->fine_rows = h->member && layers == 1 ? ensemble_tile_rows(h->esz)
                                                : (int)fine_tile_rows(h->esz);
        h->fine_ry = fine_rows_per_thread(levels);
        guard(fine_maps(h));
    }
    if (s == QG_OK) guard(dev_alloc(h, (void**)&h->dpart, sizeof(double) * 5 * diag_blocks()));
    if (s == QG_OK) guard(dev_alloc(h, (void**)&h->dout, sizeof(double) * 8));
    if (s == QG_OK && cudaMallocHost((void**)&h->hout, sizeof(double) * 8) != cudaSuccess) guard(QG_ERR_OOM);
    if (s == QG_OK) {
        const double pi = 3.14159265358979323846;
        std::vector<double> fr(h->ny + 1, 0.0);
        for (int j = 1; j < h->ny; ++j) {
            const double y = h->y0 + h->dy * j;
            fr[j] = layers == 1 ? h->amp * std::sin(pi * y) / Ro : h->amp * std::sin(2.0 * pi * y);
        }
        guard(upload_real(h, &h->frow, fr));
    }
    if (s == QG_OK) {
        const LevelTables* t = nullptr;
        guard(get_level(h, levels, &t));
    }
    if (s == QG_OK && cudaDeviceSynchronize() != cudaSuccess) guard(QG_ERR_CUDA);
    if (s == QG_OK)
        guard(h->dtype == QG_F64 ? autotune_solve<double>(h) : autotune_solve<float>(h));
    if (s != QG_OK) {
        qg_destroy(h);
        (void)cudaGetLastError();
        return s;
    }
    *out = h;
    return QG_OK;
}

static void tape_release(qg_ctx* h);

qg_status qg_destroy(qg_handle h) {
    if (!h) return QG_OK;
    cudaStreamSynchronize(h->stream);
    for (cudaStream_t x : {h->xin, h->xout}) {
        if (!x) continue;
        cudaStreamSynchronize(x);
        cudaStreamDestroy(x);
    }
    for (int b = 0; b < 2; ++b)
        for (cudaEvent_t e : {h->in_ready[b], h->in_free[b], h->out_ready[b], h->out_free[b]})
            if (e) cudaEventDestroy(e);
    tape_release(h);
    drop_graph(h);
    for (void* p : h->allocs) cudaFree(p);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->hout) cudaFreeHost(h->hout);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    delete h;
    return QG_OK;
}

qg_status qg_last_error(qg_handle h) {
    if (!h) return QG_ERR_ARG;
    qg_status s = h->latched;
    h->latched = QG_OK;
    return s;
}

// Reads and clears the device error flag of the bounded waits.
static qg_status check_device_flag(qg_ctx* h) {
    int flag = 0;
    QG_TRY(cudaMemcpyAsync(&flag, h->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    QG_TRY(cudaStreamSynchronize(h->stream));
    if (flag) {
        QG_TRY(cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream));
        QG_TRY(cudaMemsetAsync(h->dbar, 0, sizeof(unsigned) * 2, h->stream));
        return fail(h, QG_ERR_TIMEOUT);
    }
    return QG_OK;
}

qg_status qg_synchronize(qg_handle h) {
    if (!h) return QG_ERR_ARG;
    QG_TRY(cudaStreamSynchronize(h->stream));
    if (h->xout) QG_TRY(cudaStreamSynchronize(h->xout));
    qg_status s = check_device_flag(h);
    if (s != QG_OK) {
        qg_last_error(h);
        return s;
    }
    return qg_last_error(h);
}

// Whether ptr is page-locked host memory (copied by DMA through staging).
static bool pinned_host(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// The transfer streams, events and staging buffers, made on first use.
static qg_status xfer_init(qg_ctx* h) {
    if (h->xin) return QG_OK;
    const size_t bytes = (size_t)(h->nx - 1) * (h->ny - 1) * h->esz;
    for (int b = 0; b < 2; ++b) {
        qg_status st = dev_alloc(h, &h->stage_in[b], bytes);
        if (st == QG_OK) st = dev_alloc(h, &h->stage_out[b], bytes);
        if (st != QG_OK) return st;
        for (cudaEvent_t* e : {&h->in_ready[b], &h->in_free[b], &h->out_ready[b], &h->out_free[b]})
            if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return QG_ERR_CUDA;
    }
    if (cudaStreamCreateWithFlags(&h->xout, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->xin, cudaStreamNonBlocking) != cudaSuccess)
        return QG_ERR_CUDA;
    return QG_OK;
}

qg_status qg_set_state(qg_handle h, const void* field, int layer) {
    NvtxRange nvtx_range("qg_set_state");
    if (!h || !field || layer < 0 || layer >= h->layers) return QG_ERR_ARG;
    if (h->latched != QG_OK) return qg_last_error(h);
    char* dst = static_cast<char*>(h->w[0]) + (size_t)layer * h->plane_f * h->esz;
    if (pinned_host(field)) {
        // DMA into a staging buffer on the upload stream (it may run while
        // earlier steps still compute), then the repack on the handle's
        // stream, which waits for the upload
        QG_TRY_S(xfer_init(h));
        const int b = h->bin;
        h->bin ^= 1;
        const size_t bytes = (size_t)(h->nx - 1) * (h->ny - 1) * h->esz;
        QG_TRY(cudaStreamWaitEvent(h->xin, h->in_free[b], 0));
        QG_TRY(cudaMemcpyAsync(h->stage_in[b], field, bytes, cudaMemcpyHostToDevice, h->xin));
        QG_TRY(cudaEventRecord(h->in_ready[b], h->xin));
        QG_TRY(cudaStreamWaitEvent(h->stream, h->in_ready[b], 0));
        QG_TRY(copy_in(dst, h->ldf, h->stage_in[b], h->nx - 1, h->ny - 1, h->esz, h->stream));
        QG_TRY(cudaEventRecord(h->in_free[b], h->stream));
    } else {
        QG_TRY(copy_in(dst, h->ldf, field, h->nx - 1, h->ny - 1, h->esz, h->stream));
    }
    h->part_valid = false;
    h->time_host = 0.0;
    if (h->solver == QG_SOLVER_MULTIGRID)   // the first solve's guess: zero
        QG_TRY(cudaMemsetAsync(h->levels ? h->cpsi : h->psi, 0,
                               (h->levels ? h->plane_c : h->plane_f) * h->esz, h->stream));
    QG_TRY(cudaMemsetAsync(h->dclock, 0, sizeof(double) * 4, h->stream));
    return QG_OK;
}

qg_status qg_get_state(qg_handle h, void* field, int layer) {
    NvtxRange nvtx_range("qg_get_state");
    if (!h || !field || layer < 0 || layer >= h->layers) return QG_ERR_ARG;
    if (h->latched != QG_OK) return qg_last_error(h);
    const char* src = static_cast<const char*>(h->w[0]) + (size_t)layer * h->plane_f * h->esz;
    QG_TRY(copy_out(field, src, h->ldf, h->nx - 1, h->ny - 1, h->esz, h->stream));
    return QG_OK;
}

qg_status qg_get_state_async(qg_handle h, void* field, int layer) {
    NvtxRange nvtx_range("qg_get_state_async");
    if (!h || !field || layer < 0 || layer >= h->layers) return QG_ERR_ARG;
    if (h->latched != QG_OK) return qg_last_error(h);
    if (!pinned_host(field)) return qg_get_state(h, field, layer);
    QG_TRY_S(xfer_init(h));
    const int b = h->bout;
    h->bout ^= 1;
    const size_t bytes = (size_t)(h->nx - 1) * (h->ny - 1) * h->esz;
    const char* src = static_cast<const char*>(h->w[0]) + (size_t)layer * h->plane_f * h->esz;
    // the repack into a staging buffer on the handle's stream (once the
    // download of two calls ago has emptied it), then the DMA to the host on
    // the download stream, which the handle's later work does not wait for
    QG_TRY(cudaStreamWaitEvent(h->stream, h->out_free[b], 0));
    QG_TRY(copy_out(h->stage_out[b], src, h->ldf, h->nx - 1, h->ny - 1, h->esz, h->stream));
    QG_TRY(cudaEventRecord(h->out_ready[b], h->stream));
    QG_TRY(cudaStreamWaitEvent(h->xout, h->out_ready[b], 0));
    QG_TRY(cudaMemcpyAsync(field, h->stage_out[b], bytes, cudaMemcpyDeviceToHost, h->xout));
    QG_TRY(cudaEventRecord(h->out_free[b], h->xout));
    return QG_OK;
}

qg_status qg_get_psi(qg_handle h, void* psi, int layer) {
    if (!h || !psi || layer < 0 || layer >= h->layers) return QG_ERR_ARG;
    if (h->latched != QG_OK) return qg_last_error(h);
    qg_status s = project_any(h, h->w[0], h->stream);
    if (s != QG_OK) return s;
    const char* src = static_cast<const char*>(h->psi) + (size_t)layer * h->plane_f * h->esz;
    QG_TRY(copy_out(psi, src, h->ldf, h->nx - 1, h->ny - 1, h->esz, h->stream));
    return QG_OK;
}

qg_status qg_set_forcing(qg_handle h, const void* forcing) {
    if (!h) return QG_ERR_ARG;
    if (h->layers != 1) return QG_ERR_UNSUPPORTED;
    if (h->latched != QG_OK) return qg_last_error(h);
    drop_graph(h);
    if (!forcing) {
        h->f2d = nullptr;   // f2d_buf stays allocated for reuse
        return QG_OK;
    }
    if (!h->f2d_buf) {
        // allocated on first use; listed in allocs so qg_destroy frees it
        void* p = nullptr;
        qg_status s = dev_alloc(h, &p, h->plane_f * h->esz);
        if (s != QG_OK) return fail(h, s);
        h->f2d_buf = p;
    }
    h->f2d = h->f2d_buf;
    if (make_tensor_map(&h->tm_f, h->f2d, h->nx, h->ny, h->ldf, h->esz, fine_block_cols(),
                        h->fine_rows) != cudaSuccess)
        return fail(h, QG_ERR_CUDA);
    QG_TRY(copy_in(h->f2d, h->ldf, forcing, h->nx - 1, h->ny - 1, h->esz, h->stream));
    return QG_OK;
}

qg_status qg_poisson_solve(qg_handle h, const void* rhs, void* psi, int level) {
    NvtxRange nvtx_range("qg_poisson_solve");
    if (!h || !rhs || !psi || level < 0 || level > h->levels) return QG_ERR_ARG;
    if (h->latched != QG_OK) return qg_last_error(h);
    if (h->solver == QG_SOLVER_MULTIGRID &&
        !mg_supports(h->nx >> level, h->ny >> level, h->dx, h->dy))
        return QG_ERR_UNSUPPORTED;
    const LevelTables* t = nullptr;
    qg_status s = get_level(h, level, &t);
    if (s != QG_OK) return fail(h, s);
    const size_t pl = (size_t)(t->my + 1) * t->ldc;
    const int ld_tr = padded_ld(t->my);
    const size_t pl_tr = (size_t)(t->mx + 1) * ld_tr;
    // (the multigrid path keeps its result in the second part)
    const size_t bytes = (pl + (pl_tr > pl ? pl_tr : pl)) * h->layers * h->esz;
    void* buf = nullptr;
    QG_TRY(cudaMallocAsync(&buf, bytes, h->stream));
    void* tbuf = static_cast<char*>(buf) + pl * h->layers * h->esz;
    cudaError_t e = cudaMemsetAsync(buf, 0, bytes, h->stream);
    const size_t dense = (size_t)(t->mx - 1) * (t->my - 1) * h->esz;
    void* buf_out = buf;
    for (int L = 0; L < h->layers && e == cudaSuccess; ++L)
        e = copy_in(static_cast<char*>(buf) + L * pl * h->esz, t->ldc,
                    static_cast<const char*>(rhs) + L * dense, t->mx - 1, t->my - 1,
                    h->esz, h->stream);
    if (e == cudaSuccess && h->solver == QG_SOLVER_MULTIGRID) {
        s = h->dtype == QG_F64
                ? mg_solve_level<double>(h, *t, buf, 1, tbuf, pl, h->stream, true)
                : mg_solve_level<float>(h, *t, buf, 1, tbuf, pl, h->stream, true);
        if (s != QG_OK) e = cudaErrorUnknown;
        buf_out = tbuf;
    } else if (e == cudaSuccess) {
        s = h->dtype == QG_F64
                ? solve_level<double>(h, *t, buf, tbuf, ld_tr, pl_tr, buf, buf, pl, h->stream)
                : solve_level<float>(h, *t, buf, tbuf, ld_tr, pl_tr, buf, buf, pl, h->stream);
        if (s != QG_OK) e = cudaErrorUnknown;
    }
    for (int L = 0; L < h->layers && e == cudaSuccess; ++L)
        e = copy_out(static_cast<char*>(psi) + L * dense,
                     static_cast<char*>(buf_out) + L * pl * h->esz,
                     t->ldc, t->mx - 1, t->my - 1, h->esz, h->stream);
    cudaFreeAsync(buf, h->stream);
    if (s != QG_OK) return s;
    QG_TRY(e);
    return QG_OK;
}

static qg_status transfer(qg_handle h, const void* src, void* dst, int levels, bool down) {
    if (!h || !src || !dst || levels < 1) return QG_ERR_ARG;
    if ((h->nx >> levels) < 2 || (h->ny >> levels) < 2) return QG_ERR_ARG;
    if (h->latched != QG_OK) return qg_last_error(h);
    const int mx = h->nx >> levels, my = h->ny >> levels, ldc = padded_ld(mx);
    const size_t bf = h->plane_f * h->esz, bc = (size_t)(my + 1) * ldc * h->esz;
    void* f = nullptr;
    void* c = nullptr;
    QG_TRY(cudaMallocAsync(&f, bf, h->stream));
    cudaError_t e = cudaMallocAsync(&c, bc, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(f, 0, bf, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c, 0, bc, h->stream);
    if (down) {
        if (e == cudaSuccess) e = copy_in(f, h->ldf, src, h->nx - 1, h->ny - 1, h->esz, h->stream);
        if (e == cudaSuccess)
            e = h->dtype == QG_F64
                    ? launch_restrict<double>((const double*)f, h->ldf, (double*)c, ldc, mx, my, levels, h->stream)
                    : launch_restrict<float>((const float*)f, h->ldf, (float*)c, ldc, mx, my, levels, h->stream);
        if (e == cudaSuccess) e = copy_out(dst, c, ldc, mx - 1, my - 1, h->esz, h->stream);
    } else {
        if (e == cudaSuccess) e = copy_in(c, ldc, src, mx - 1, my - 1, h->esz, h->stream);
        if (e == cudaSuccess)
            e = h->dtype == QG_F64
                    ? launch_prolong<double>((const double*)c, ldc, (double*)f, h->ldf, h->nx, h->ny, levels, h->stream)
                    : launch_prolong<float>((const float*)c, ldc, (float*)f, h->ldf, h->nx, h->ny, levels, h->stream);
        if (e == cudaSuccess) e = copy_out(dst, f, h->ldf, h->nx - 1, h->ny - 1, h->esz, h->stream);
    }
    if (c) cudaFreeAsync(c, h->stream);
    cudaFreeAsync(f, h->stream);
    QG_TRY(e);
    return QG_OK;
}

qg_status qg_restrict(qg_handle h, const void* fine, void* coarse, int levels) {
    NvtxRange nvtx_range("qg_restrict");
    return transfer(h, fine, coarse, levels, true);
}

qg_status qg_prolong(qg_handle h, const void* coarse, void* fine, int levels) {
    NvtxRange nvtx_range("qg_prolong");
    return transfer(h, coarse, fine, levels, false);
}

qg_status qg_step(qg_handle h, int64_t n) {
    NvtxRange nvtx_range("qg_step");
    if (!h || n < 0) return QG_ERR_ARG;
    if (h->latched != QG_OK) return qg_last_error(h);
    if (n == 0) return QG_OK;
    qg_status s = build_graph(h);
    if (s != QG_OK) return s;
    if (h->part && !h->part_valid) {
        s = h->dtype == QG_F64 ? init_partials<double>(h, h->stream) : init_partials<float>(h, h->stream);
        if (s != QG_OK) return s;
        h->part_valid = true;
    }
    Tape* tp = h->tape;
    if (tp && (tp->reversing || tp->recorded + n > tp->max_steps)) return QG_ERR_ARG;
    if (h->layers == 2) h->time_host += (double)n * h->dt;
    if (h->stats) h->stat_count += n;
    const size_t bytes = h->plane_f * h->esz;
    for (int64_t k = 0; k < n; ++k) {
        QG_TRY(cudaGraphLaunch(h->gexec, h->stream));
        if (tp) {
            ++tp->recorded;
            tp->cursor = tp->recorded;
            if (tp->recorded % tp->every == 0)
                QG_TRY(cudaMemcpyAsync(tp->ckpt[tp->recorded / tp->every], h->w[0], bytes,
                                       cudaMemcpyDeviceToDevice, h->stream));
        }
    }
    return QG_OK;
}

qg_status qg_set_timing(qg_handle h, int enable) {
    if (!h) return QG_ERR_ARG;
    return qg_set_timing_mask(h, enable ? ~0u : 0u);
}

qg_status qg_set_timing_mask(qg_handle h, uint32_t mask) {
    if (!h) return QG_ERR_ARG;
    const bool on = mask != 0;
    if (on != h->timing || (on && mask != h->timing_mask)) {
        QG_TRY(cudaStreamSynchronize(h->stream));
        drop_graph(h);
        h->timing = on;
        h->timing_mask = on ? mask : ~0u;
    }
    return QG_OK;
}

qg_status qg_set_cfl(qg_handle h, double c) {
    if (!h || !(c >= 0.0) || !std::isfinite(c)) return QG_ERR_ARG;
    // Eq. dt is stated for Courant numbers c <= 1 (Section 4.2)
    if (c > 1.0) return QG_ERR_CFL;
    if (c > 0.0 && (h->layers != 1 || h->tape)) return QG_ERR_UNSUPPORTED;
    if (c != h->cfl) {
        QG_TRY(cudaStreamSynchronize(h->stream));
        drop_graph(h);
        h->cfl = c;
    }
    return QG_OK;
}

qg_status qg_set_solver(qg_handle h, qg_solver kind, int32_t cycles) {
    if (!h || (kind != QG_SOLVER_FFT && kind != QG_SOLVER_MULTIGRID)) return QG_ERR_ARG;
    if (kind == QG_SOLVER_MULTIGRID) {
        if (cycles < 1 || cycles > 64) return QG_ERR_ARG;
        if (h->layers != 1 || h->tape ||
            !mg_supports(h->nx >> h->levels, h->ny >> h->levels, h->dx, h->dy))
            return QG_ERR_UNSUPPORTED;
    }
    if (h->latched != QG_OK) return qg_last_error(h);
    QG_TRY(cudaStreamSynchronize(h->stream));
    if (kind == QG_SOLVER_MULTIGRID) {
        // the hierarchy of the step's grid now: no allocation during capture
        const MGPlan* mp = nullptr;
        qg_status s = get_mg(h, h->nx >> h->levels, h->ny >> h->levels, &mp);
        if (s != QG_OK) return s;
    }
    drop_graph(h);
    h->solver = kind;
    if (kind == QG_SOLVER_MULTIGRID) {
        h->mg_cycles = cycles;
        QG_TRY(cudaMemsetAsync(h->levels ? h->cpsi : h->psi, 0,
                               (h->levels ? h->plane_c : h->plane_f) * h->esz, h->stream));
    }
    return QG_OK;
}

qg_status qg_get_time(qg_handle h, double* t, double* dt_last) {
    if (!h) return QG_ERR_ARG;
    if (h->latched != QG_OK) return qg_last_error(h);
    double v[4] = {0, 0, 0, 0};
    if (h->layers == 1) {
        QG_TRY(cudaMemcpyAsync(v, h->dclock, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
        QG_TRY(cudaStreamSynchronize(h->stream));
    } else {
        QG_TRY(cudaStreamSynchronize(h->stream));
        v[1] = h->time_host;
        v[2] = h->dt;
    }
    if (t) *t = v[1];
    if (dt_last) *dt_last = v[2];
    return QG_OK;
}

qg_status qg_stats_begin(qg_handle h) {
    if (!h) return QG_ERR_ARG;
    if (h->tape) return QG_ERR_UNSUPPORTED;
    if (h->latched != QG_OK) return qg_last_error(h);
    const bool fine = h->levels == 0;
    const size_t n = (fine ? h->plane_f : h->plane_c) * h->layers;
    const size_t nw = h->plane_f * h->layers;
    if (!h->stat_acc) {
        qg_status s = dev_alloc(h, (void**)&h->stat_acc, n * sizeof(double));
        if (s != QG_OK) return s;
    }
    if (!h->stat_acc_w) {
        qg_status s = dev_alloc(h, (void**)&h->stat_acc_w, nw * sizeof(double));
        if (s != QG_OK) return s;
    }
    QG_TRY(cudaMemsetAsync(h->stat_acc, 0, n * sizeof(double), h->stream));
    QG_TRY(cudaMemsetAsync(h->stat_acc_w, 0, nw * sizeof(double), h->stream));
    h->stat_count = 0;
    if (!h->stats) {
        QG_TRY(cudaStreamSynchronize(h->stream));
        drop_graph(h);
        h->stats = true;
    }
    return QG_OK;
}

qg_status qg_stats_mean_psi(qg_handle h, void* psi_mean, int layer, int64_t* count) {
    NvtxRange nvtx_range("qg_stats_mean_psi");
    if (!h || layer < 0 || layer >= h->layers) return QG_ERR_ARG;
    if (!h->stats || h->stat_count == 0) return QG_ERR_ARG;
    if (h->latched != QG_OK) return qg_last_error(h);
    if (count) *count = h->stat_count;
    if (!psi_mean) return QG_OK;
    const double sc = 1.0 / (double)h->stat_count;
    const bool fine = h->levels == 0;
    const LevelTables* t = nullptr;
    qg_status st = get_level(h, h->levels, &t);
    if (st != QG_OK) return st;
    const double* acc = h->stat_acc + (size_t)layer * (fine ? h->plane_f : h->plane_c);
    const int ld = fine ? h->ldf : t->ldc;
    const int lv = fine ? 0 : h->levels;
    if (h->dtype == QG_F64)
        QG_TRY(launch_mean_out<double>(static_cast<double*>(psi_mean), acc, ld, sc, h->nx, h->ny,
                                       lv, h->stream));
    else
        QG_TRY(launch_mean_out<float>(static_cast<float*>(psi_mean), acc, ld, sc, h->nx, h->ny,
                                      lv, h->stream));
    return QG_OK;
}

qg_status qg_stats_mean_q(qg_handle h, void* q_mean, int layer, int64_t* count) {
    NvtxRange nvtx_range("qg_stats_mean_q");
    if (!h || layer < 0 || layer >= h->layers) return QG_ERR_ARG;
    if (!h->stats || h->stat_count == 0) return QG_ERR_ARG;
    if (h->latched != QG_OK) return qg_last_error(h);
    if (count) *count = h->stat_count;
    if (!q_mean) return QG_OK;
    // one layer: q = Ro w + y (Eq. pv); two layers: q_i = Q_i + y
    const double sc = (h->layers == 1 ? h->Ro : 1.0) / (double)h->stat_count;
    const double* acc = h->stat_acc_w + (size_t)layer * h->plane_f;
    if (h->dtype == QG_F64)
        QG_TRY(launch_mean_q_out<double>(static_cast<double*>(q_mean), acc, h->ldf, sc, h->nx,
                                         h->ny, h->y0, h->dy, h->stream));
    else
        QG_TRY(launch_mean_q_out<float>(static_cast<float*>(q_mean), acc, h->ldf, sc, h->nx,
                                        h->ny, h->y0, h->dy, h->stream));
    return QG_OK;
}

qg_status qg_stats_end(qg_handle h) {
    if (!h) return QG_ERR_ARG;
    if (h->stats) {
        QG_TRY(cudaStreamSynchronize(h->stream));
        drop_graph(h);
        h->stats = false;
    }
    return QG_OK;
}

qg_status qg_inject_fault(qg_handle h, int kind) {
    if (!h || kind < QG_FAULT_NONE || kind > QG_FAULT_BARRIER_STALL) return QG_ERR_ARG;
    if (kind != h->fault) {
        QG_TRY(cudaStreamSynchronize(h->stream));
        drop_graph(h);
        h->fault = kind;
    }
    return QG_OK;
}

qg_status qg_read_timing(qg_handle h, double* ms, int32_t* launches) {
    if (!h || !ms || !launches) return QG_ERR_ARG;
    if (!h->timing || !h->gexec) return QG_ERR_ARG;
    QG_TRY(cudaStreamSynchronize(h->stream));
    for (int c = 0; c < QG_K_COUNT; ++c) {
        ms[c] = 0.0;
        launches[c] = 0;
    }
    for (auto& u : h->ev_used) {
        float t = 0.f;
        QG_TRY(cudaEventElapsedTime(&t, u.second.first, u.second.second));
        ms[u.first] += t;
        launches[u.first] += 1;
    }
    return QG_OK;
}

qg_status qg_solve_engine(qg_handle h, int32_t* engine) {
    if (!h || !engine) return QG_ERR_ARG;
    *engine = h->solver == QG_SOLVER_MULTIGRID ? 0 : h->solve_engine;
    return QG_OK;
}

}  // extern "C"

namespace qg {
// error words of the multigrid, diagnostics and adjoint translation units
int bounds_site_mg();
int bounds_site_diag();
int bounds_site_adjoint();
}  // namespace qg

extern "C" {

qg_status qg_bounds_check_result(int32_t* site) {
    if (!site) return QG_ERR_ARG;
#ifdef QG_BOUNDS_CHECK
    if (cudaDeviceSynchronize() != cudaSuccess) {
        (void)cudaGetLastError();
        return QG_ERR_CUDA;
    }
    int first = 0;
    for (int v : {bounds_site_fused(), bounds_site_solve32(), bounds_site_stencil(),
                  bounds_site_mtx(), bounds_site_stream(), bounds_site_tc(), qg::bounds_site_mg(),
                  qg::bounds_site_diag(), qg::bounds_site_adjoint()}) {
        if (v < 0) return QG_ERR_CUDA;
        if (!first) first = v;
    }
    *site = first;
    return QG_OK;
#else
    *site = 0;
    return QG_ERR_UNSUPPORTED;
#endif
}

qg_status qg_stencil_tile(qg_handle h, int32_t* rows, int32_t* rows_per_thread) {
    if (!h || !rows) return QG_ERR_ARG;
    *rows = h->fine_rows;
    if (rows_per_thread) *rows_per_thread = h->fine_ry;
    return QG_OK;
}

qg_status qg_step_kernel_count(qg_handle h, int64_t* count) {
    if (!h || !count) return QG_ERR_ARG;
    qg_status s = build_graph(h);
    if (s != QG_OK) return s;
    *count = h->kernels_per_step;
    return QG_OK;
}

qg_status qg_diagnostics(qg_handle h, double* ke, double* enstrophy, double* max_vel) {
    NvtxRange nvtx_range("qg_diagnostics");
    if (!h) return QG_ERR_ARG;
    if (h->latched != QG_OK) return qg_last_error(h);
    qg_status s = project_any(h, h->w[0], h->stream);
    if (s != QG_OK) return s;
    if (h->dtype == QG_F64)
        QG_TRY(launch_diagnostics<double>((const double*)h->psi, (const double*)h->w[0], h->nx,
                                          h->ny, h->ldf, h->dx, h->dy, h->dpart, diag_blocks(),
                                          h->dout, h->stream));
    else
        QG_TRY(launch_diagnostics<float>((const float*)h->psi, (const float*)h->w[0], h->nx,
                                         h->ny, h->ldf, h->dx, h->dy, h->dpart, diag_blocks(),
                                         h->dout, h->stream));
    QG_TRY(cudaMemcpyAsync(h->hout, h->dout, sizeof(double) * 5, cudaMemcpyDeviceToHost, h->stream));
    QG_TRY(cudaStreamSynchronize(h->stream));
    {
        const qg_status fs = check_device_flag(h);
        if (fs != QG_OK) return fs;
    }
    const double* r = h->hout;
    const double dx = h->dx, dy = h->dy;
    const double E = 0.5 * dx * dy * (r[0] / (dx * dx) + r[1] / (dy * dy));
    const double Z = 0.5 * dx * dy * r[2];
    const double U = std::fmax(r[3] / (2.0 * dx), r[4] / (2.0 * dy));
    if (!std::isfinite(E) || !std::isfinite(Z)) return fail(h, QG_ERR_NONFINITE);
    if (ke) *ke = E;
    if (enstrophy) *enstrophy = Z;
    if (max_vel) *max_vel = U;
    return QG_OK;
}

qg_status qg_energy_accumulate(qg_handle h, double scale, double* acc) {
    NvtxRange nvtx_range("qg_energy_accumulate");
    if (!h || !acc || !std::isfinite(scale)) return QG_ERR_ARG;
    if (h->latched != QG_OK) return qg_last_error(h);
    qg_status s = project_any(h, h->w[0], h->stream);
    if (s != QG_OK) return s;
    if (h->dtype == QG_F64)
        QG_TRY(launch_diagnostics<double>((const double*)h->psi, (const double*)h->w[0], h->nx,
                                          h->ny, h->ldf, h->dx, h->dy, h->dpart, diag_blocks(),
                                          h->dout, h->stream));
    else
        QG_TRY(launch_diagnostics<float>((const float*)h->psi, (const float*)h->w[0], h->nx,
                                         h->ny, h->ldf, h->dx, h->dy, h->dpart, diag_blocks(),
                                         h->dout, h->stream));
    // E = 1/2 dx dy (sx/dx^2 + sy/dy^2), as qg_diagnostics forms it
    const double c0 = scale * 0.5 * h->dy / h->dx, c1 = scale * 0.5 * h->dx / h->dy;
    QG_TRY(launch_energy_add(h->dout, c0, c1, acc, h->stream));
    return QG_OK;
}

}  // extern "C"

// ---- adjoint ---------------------------------------------------------------

namespace {

void tape_free_all(Tape* tp) {
    for (void* p : tp->allocs) cudaFree(p);
    delete tp;
}

template <typename T>
StageParams<T> stage_params(const qg_ctx* h, double a, double b) {
    StageParams<T> p;
    p.nx = h->nx;
    p.ny = h->ny;
    p.ld = h->ldf;
    p.c_jac = (T)(1.0 / (12.0 * h->dx * h->dy));
    p.c_beta = (T)(1.0 / (12.0 * h->Ro * h->dx));
    p.c_lapx = (T)(1.0 / (h->Re * h->dx * h->dx));
    p.c_lapy = (T)(1.0 / (h->Re * h->dy * h->dy));
    p.dt = (T)h->dt;
    p.a = (T)a;
    p.b = (T)b;
    return p;
}

template <typename T>
AdjParams<T> adj_params(const qg_ctx* h, double a, double b) {
    AdjParams<T> p;
    p.nx = h->nx;
    p.ny = h->ny;
    p.ld = h->ldf;
    p.c_jac = (T)(1.0 / (12.0 * h->dx * h->dy));
    p.c_beta = (T)(1.0 / (12.0 * h->Ro * h->dx));
    p.c_lapx = (T)(1.0 / (h->Re * h->dx * h->dx));
    p.c_lapy = (T)(1.0 / (h->Re * h->dy * h->dy));
    p.dt = (T)h->dt;
    p.a = (T)a;
    p.b = (T)b;
    p.inv_dx2 = (T)(1.0 / (h->dx * h->dx));
    p.inv_dy2 = (T)(1.0 / (h->dy * h->dy));
    p.dxdy = (T)(h->dx * h->dy);
    return p;
}

// The forward state at tape time t (t <= recorded).
template <typename T>
qg_status tape_state(qg_ctx* h, int64_t t, const void** out) {
    Tape* tp = h->tape;
    const size_t bytes = h->plane_f * h->esz;
    if (tp->every == 1) {
        *out = tp->ckpt[t];
        return QG_OK;
    }
    const int64_t start = t / tp->every * tp->every;
    if (tp->seg_start != start) {
        if (!tp->live) {
            QG_TRY(cudaMalloc(&tp->live, bytes + 4 * sizeof(double)));
            tp->allocs.push_back(tp->live);
            QG_TRY(cudaMemcpyAsync(tp->live, h->w[0], bytes, cudaMemcpyDeviceToDevice, h->stream));
            QG_TRY(cudaMemcpyAsync(static_cast<char*>(tp->live) + bytes, h->dclock,
                                   4 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        }
        void* c = tp->ckpt[start / tp->every];
        QG_TRY(cudaMemcpyAsync(tp->seg[0], c, bytes, cudaMemcpyDeviceToDevice, h->stream));
        QG_TRY(cudaMemcpyAsync(h->w[0], c, bytes, cudaMemcpyDeviceToDevice, h->stream));
        qg_status s = build_graph(h);
        if (s != QG_OK) return s;
        if (h->part) {
            s = init_partials<T>(h, h->stream);
            if (s != QG_OK) return s;
        }
        const int64_t end = std::min(start + tp->every, tp->recorded);
        for (int64_t k = 1; k <= end - start; ++k) {
            QG_TRY(cudaGraphLaunch(h->gexec, h->stream));
            QG_TRY(cudaMemcpyAsync(tp->seg[k], h->w[0], bytes, cudaMemcpyDeviceToDevice, h->stream));
        }
        h->part_valid = false;
        tp->seg_start = start;
    }
    *out = tp->seg[t - start];
    return QG_OK;
}

// lam(t) -> lam(t - 1) through the step from w^n = w (tape time t - 1): the
// three stages are recomputed (w^(1), w^(2), psi^(0..2)), then reversed.
template <typename T>
qg_status adjoint_one(qg_ctx* h, const void* w) {
    Tape* tp = h->tape;
    cudaStream_t s = h->stream;
    T* B[Tape::NBUF];
    for (int k = 0; k < Tape::NBUF; ++k) B[k] = static_cast<T*>(tp->buf[k]);
    const T* wn = static_cast<const T*>(w);
    const T* frow = static_cast<const T*>(h->frow);
    const T* f2d = static_cast<const T*>(h->f2d);
    static const double RA[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double RB[3] = {1.0, 0.25, 2.0 / 3.0};
    // forward stages
    qg_status st = project_to<T>(h, wn, B[Tape::P0], s);
    if (st != QG_OK) return st;
    QG_TRY(launch_fine_stage<T>(B[Tape::P0], wn, wn, B[Tape::W1], frow, f2d,
                                stage_params<T>(h, RA[0], RB[0]), s));
    if ((st = project_to<T>(h, B[Tape::W1], B[Tape::P1], s)) != QG_OK) return st;
    QG_TRY(launch_fine_stage<T>(B[Tape::P1], B[Tape::W1], wn, B[Tape::W2], frow, f2d,
                                stage_params<T>(h, RA[1], RB[1]), s));
    if ((st = project_to<T>(h, B[Tape::W2], B[Tape::P2], s)) != QG_OK) return st;
    // reverse: lam in L0, result in ACC
    QG_TRY(cudaMemsetAsync(B[Tape::ACC], 0, h->plane_f * h->esz, s));
    const T* ws[3] = {wn, B[Tape::W1], B[Tape::W2]};
    const T* ps[3] = {B[Tape::P0], B[Tape::P1], B[Tape::P2]};
    T* lam = B[Tape::L0];
    T* nxt = B[Tape::L1];
    for (int k = 2; k >= 0; --k) {
        const AdjParams<T> p = adj_params<T>(h, RA[k], RB[k]);
        QG_TRY(launch_adj_source<T>(ws[k], lam, B[Tape::U], p, s));
        if ((st = project_to<T>(h, B[Tape::U], B[Tape::PHI], s)) != QG_OK) return st;
        T* out = k == 0 ? B[Tape::ACC] : nxt;
        QG_TRY(launch_adj_stage<T>(ps[k], lam, B[Tape::PHI], out, B[Tape::ACC], B[Tape::GF], p,
                                   k == 0, s));
        if (k > 0) std::swap(lam, nxt);
    }
    std::swap(tp->buf[Tape::L0], tp->buf[Tape::ACC]);
    return QG_OK;
}

template <typename T>
qg_status adjoint_steps(qg_ctx* h, int64_t n, void* lambda, void* dJdF) {
    Tape* tp = h->tape;
    cudaStream_t s = h->stream;
    const size_t bytes = h->plane_f * h->esz;
    tp->reversing = true;
    QG_TRY(copy_in(tp->buf[Tape::L0], h->ldf, lambda, h->nx - 1, h->ny - 1, h->esz, s));
    QG_TRY(cudaMemsetAsync(tp->buf[Tape::GF], 0, bytes, s));
    for (int64_t k = 0; k < n; ++k) {
        const void* w = nullptr;
        qg_status st = tape_state<T>(h, tp->cursor - 1, &w);
        if (st != QG_OK) return st;
        if ((st = adjoint_one<T>(h, w)) != QG_OK) return st;
        --tp->cursor;
    }
    QG_TRY(copy_out(lambda, tp->buf[Tape::L0], h->ldf, h->nx - 1, h->ny - 1, h->esz, s));
    QG_TRY(launch_add_to_dense<T>(static_cast<T*>(dJdF), static_cast<const T*>(tp->buf[Tape::GF]),
                                  1.0, h->nx, h->ny, h->ldf, s));
    return QG_OK;
}

template <typename T>
qg_status energy_gradient(qg_ctx* h, double scale, void* g) {
    Tape* tp = h->tape;
    cudaStream_t s = h->stream;
    const void* w = nullptr;
    qg_status st = tape_state<T>(h, tp->cursor, &w);
    if (st != QG_OK) return st;
    T* P = static_cast<T*>(tp->buf[Tape::P0]);
    T* U = static_cast<T*>(tp->buf[Tape::U]);
    T* PHI = static_cast<T*>(tp->buf[Tape::PHI]);
    if ((st = project_to<T>(h, w, P, s)) != QG_OK) return st;
    QG_TRY(launch_energy_source<T>(P, U, adj_params<T>(h, 0.0, 0.0), s));
    if ((st = project_to<T>(h, U, PHI, s)) != QG_OK) return st;
    QG_TRY(launch_add_to_dense<T>(static_cast<T*>(g), PHI, scale, h->nx, h->ny, h->ldf, s));
    return QG_OK;
}

}  // namespace

static void tape_release(qg_ctx* h) {
    if (!h->tape) return;
    cudaStreamSynchronize(h->stream);
    tape_free_all(h->tape);
    h->tape = nullptr;
}

extern "C" {

qg_status qg_tape_begin(qg_handle h, int64_t every, int64_t max_steps) {
    if (!h || every < 1 || max_steps < 1) return QG_ERR_ARG;
    if (h->layers != 1 || h->cfl > 0.0 || h->stats || h->solver != QG_SOLVER_FFT)
        return QG_ERR_UNSUPPORTED;
    if (h->latched != QG_OK) return qg_last_error(h);
    tape_release(h);
    Tape* tp = new (std::nothrow) Tape();
    if (!tp) return QG_ERR_OOM;
    tp->every = every;
    tp->max_steps = max_steps;
    const size_t bytes = h->plane_f * h->esz;
    auto alloc = [&](void** p) {
        if (cudaMalloc(p, bytes) != cudaSuccess) return false;
        tp->allocs.push_back(*p);
        return cudaMemsetAsync(*p, 0, bytes, h->stream) == cudaSuccess;
    };
    bool ok = true;
    const int64_t nck = max_steps / every + 1;
    for (int64_t k = 0; k < nck && ok; ++k) {
        void* p = nullptr;
        ok = alloc(&p);
        if (ok) tp->ckpt.push_back(p);
    }
    for (int64_t k = 0; every > 1 && k <= every && ok; ++k) {
        void* p = nullptr;
        ok = alloc(&p);
        if (ok) tp->seg.push_back(p);
    }
    for (int k = 0; k < Tape::NBUF && ok; ++k) ok = alloc(&tp->buf[k]);
    if (ok) ok = cudaMemcpyAsync(tp->ckpt[0], h->w[0], bytes, cudaMemcpyDeviceToDevice,
                                 h->stream) == cudaSuccess;
    if (!ok) {
        cudaStreamSynchronize(h->stream);
        tape_free_all(tp);
        (void)cudaGetLastError();
        return QG_ERR_OOM;
    }
    h->tape = tp;
    return QG_OK;
}

qg_status qg_tape_end(qg_handle h) {
    if (!h) return QG_ERR_ARG;
    Tape* tp = h->tape;
    if (!tp) return QG_OK;
    if (tp->live) {
        const size_t bytes = h->plane_f * h->esz;
        QG_TRY(cudaMemcpyAsync(h->w[0], tp->live, bytes, cudaMemcpyDeviceToDevice, h->stream));
        QG_TRY(cudaMemcpyAsync(h->dclock, static_cast<const char*>(tp->live) + bytes,
                               4 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        h->part_valid = false;
    }
    tape_release(h);
    return QG_OK;
}

qg_status qg_adjoint_step(qg_handle h, int64_t n, void* lambda, void* dJdF) {
    NvtxRange nvtx_range("qg_adjoint_step");
    if (!h || !lambda || !dJdF || !h->tape || n < 0 || n > h->tape->cursor) return QG_ERR_ARG;
    if (h->latched != QG_OK) return qg_last_error(h);
    if (n == 0) return QG_OK;
    return h->dtype == QG_F64 ? adjoint_steps<double>(h, n, lambda, dJdF)
                              : adjoint_steps<float>(h, n, lambda, dJdF);
}

qg_status qg_energy_gradient(qg_handle h, double scale, void* g) {
    if (!h || !g || !h->tape) return QG_ERR_ARG;
    if (h->latched != QG_OK) return qg_last_error(h);
    return h->dtype == QG_F64 ? energy_gradient<double>(h, scale, g)
                              : energy_gradient<float>(h, scale, g);
}

}  // extern "C"

// ---- ensembles -------------------------------------------------------------
// One ensemble step is one CUDA graph.  Members whose elliptic grids have the
// same shape and spacings (so the same solver tables) form a group; members
// of different groups never interact, so each group's three TVDRK3 stages
// run as one chain on a branch of its own, beside the other groups:
//   * one solve launch per stage for the whole group: the warp-group FFT
//     engine as a work queue over the slots of all members (no grid
//     barriers, so groups can share the GPU), or the matrix form with one
//     CTA per member; each member's right-hand side, arrays and error flag
//     come from a device table.  A group that cannot batch (multigrid, or a
//     non-batching engine forced through QG_SOLVE_ENGINE) solves member by
//     member with the handles' own launches;
//   * the per-member extras of the first stage (time-mean accumulation, the
//     maximum velocity of Eq. dt);
//   * one fused fine-stage launch per CGP level among the group's members,
//     over all their tiles, each CTA reading its member's tensor maps and
//     parameters from a device table.
// Within a branch the launches follow each other with programmatic
// dependent launch, as in a single basin's step.

#define QG_TRY_E(expr)                        \
    do {                                      \
        const qg_status qg_s_ = (expr);       \
        if (qg_s_ != QG_OK) return qg_s_;     \
    } while (0)

// Programmatic dependent launch inside a group's branch: off, because a
// dependent kernel that starts early holds SM resources idle in its wait
// while the other branches have work for them.
constexpr bool kEnsemblePdl = false;

struct EnsFineGroup {
    int lv = 0;
    bool f2d = false;                 // some member uses a forcing field
    std::vector<int> members;
    void* dmem = nullptr;             // FineMember<T>[3 stages][members]
    int4* dtiles = nullptr;
    int ntiles = 0;
};

struct EnsSolveGroup {
    int mx = 0, my = 0, engine = 0;   // engine 0: the members solve on their own
    double dxc = 0, dyc = 0;
    std::vector<int> members;
    void* dmem = nullptr;             // SolveMember<T>[3 stages][members]
    unsigned* dq = nullptr;           // work-queue counters of the batched solve
    std::vector<EnsFineGroup> fine;   // the members by CGP level
};

struct qg_ensemble_s {
    std::vector<qg_ctx*> m;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;             // capture origin
    std::vector<cudaStream_t> lanes;        // one branch per group
    std::vector<cudaEvent_t> ev;            // fork event, then one join event per lane
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<uint64_t> gen;              // members' graph_gen when it was captured
    std::vector<EnsSolveGroup> sg;
    std::vector<void*> dallocs;             // device tables of the batched launches
    int64_t kernels = 0;
    bool fresh = false;                     // members hold no user state yet
};

namespace {

void ensemble_tables_free(qg_ensemble e) {
    for (void* p : e->dallocs) cudaFree(p);
    e->dallocs.clear();
    e->sg.clear();
}

void ensemble_free(qg_ensemble e) {
    if (!e) return;
    if (e->stream) cudaStreamSynchronize(e->stream);
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    if (e->graph) cudaGraphDestroy(e->graph);
    ensemble_tables_free(e);
    for (qg_ctx* h : e->m) qg_destroy(h);
    for (cudaEvent_t v : e->ev) cudaEventDestroy(v);
    for (cudaStream_t s : e->lanes) cudaStreamDestroy(s);
    if (e->cap) cudaStreamDestroy(e->cap);
    delete e;
}

// At least n branch streams and n + 1 events.
qg_status ensemble_lanes(qg_ensemble e, size_t n) {
    while (e->lanes.size() < n) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return QG_ERR_CUDA;
        e->lanes.push_back(s);
    }
    while (e->ev.size() < n + 1) {
        cudaEvent_t v = nullptr;
        if (cudaEventCreateWithFlags(&v, cudaEventDisableTiming) != cudaSuccess) return QG_ERR_CUDA;
        e->ev.push_back(v);
    }
    return QG_OK;
}

qg_status ens_alloc(qg_ensemble e, void** p, size_t bytes) {
    *p = nullptr;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return QG_ERR_OOM;
    }
    e->dallocs.push_back(*p);
    return QG_OK;
}

// The engines a group of members can solve with in one launch (three for
// engine 50): the warp-group FFT engines, the matrix form and engine 50
// where they take the group's grid;
// none when a member uses the multigrid solver.  An engine forced through
// QG_SOLVE_ENGINE is the only candidate, and none when it does not batch
// (then every member solves as a handle of its own would).
std::vector<int> batch_engines(qg_ensemble e, const EnsSolveGroup& g) {
    std::vector<int> out;
    for (int i : g.members)
        if (e->m[i]->solver != QG_SOLVER_FFT) return out;
    qg_ctx* h0 = e->m[g.members[0]];
    const LevelTables* t = nullptr;
    if (get_level(h0, h0->levels, &t) != QG_OK) return out;
    const int own = h0->solve_engine;
    if (h0->engine_forced) {
        if ((is_warp_engine(own) || own == kMatrixEngine || own == kTcEngine ||
             own == kStreamEngine) &&
            engine_ok(h0, t, h0->esz, own))
            out.push_back(own);
        return out;
    }
    for (int cand : {34, 33, 32, (int)kMatrixEngine, (int)kTcEngine, (int)kStreamEngine})
        if (engine_ok(h0, t, h0->esz, cand)) out.push_back(cand);
    return out;
}

template <typename T>
FusedParams<T> fused_params(qg_ctx* h, int s_idx, const LevelTables& t) {
    static const double A[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double B[3] = {1.0, 0.25, 2.0 / 3.0};
    FusedParams<T> p = {};
    p.nx = h->nx;
    p.ny = h->ny;
    p.ld = h->ldf;
    p.psi = static_cast<const T*>(h->levels == 0 ? h->psi : h->cpsi);
    p.ldp = h->levels == 0 ? h->ldf : t.ldc;
    p.w = static_cast<const T*>(h->w[s_idx]);
    p.wn = static_cast<const T*>(h->w[0]);
    p.wout = static_cast<T*>(h->w[(s_idx + 1) % 3]);
    p.frow = static_cast<const T*>(h->frow);
    p.f2d = static_cast<const T*>(h->f2d);
    for (int q = 0; q < 4; ++q) p.part[q] = h->part ? plane<T>(h->part, h->plane_c, q) : nullptr;
    p.ldc = t.ldc;
    p.err = h->derr;
    p.c_jac = (T)(1.0 / (12.0 * h->dx * h->dy));
    p.c_beta = (T)(1.0 / (12.0 * h->Ro * h->dx));
    p.c_lapx = (T)(1.0 / (h->Re * h->dx * h->dx));
    p.c_lapy = (T)(1.0 / (h->Re * h->dy * h->dy));
    p.dt = (T)h->dt;
    p.a = (T)A[s_idx];
    p.b = (T)B[s_idx];
    p.psi_o = nullptr;
    p.inv_Ro = p.k_p = p.drag = T(0);
    p.umax = h->cfl > 0.0 ? reinterpret_cast<const unsigned long long*>(h->dclock) : nullptr;
    p.cfl_h = h->cfl * std::fmin(h->dx, h->dy);
    p.dt_cap = h->dt;
    p.clock = h->dclock + 1;
    p.last_stage = s_idx == 2;
    return p;
}

template <typename T>
qg_status tune_group(qg_ensemble e, EnsSolveGroup& g, const std::vector<int>& cands,
                     bool* timed);
qg_status rest_buffers(qg_ctx* h, cudaStream_t s);

// Group the members and upload the tables of the batched launches.
template <typename T>
qg_status ensemble_tables(qg_ensemble e) {
    ensemble_tables_free(e);
    const int n = (int)e->m.size();
    // members, largest first: big tiles start first, small ones fill the tail
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (double)e->m[a]->nx * e->m[a]->ny > (double)e->m[b]->nx * e->m[b]->ny;
    });
    for (int i : order) {
        qg_ctx* h = e->m[i];
        const LevelTables* t = nullptr;
        qg_status st = get_level(h, h->levels, &t);
        if (st != QG_OK) return st;
        EnsSolveGroup* g = nullptr;
        for (auto& c : e->sg)
            if (c.mx == t->mx && c.my == t->my && c.dxc == t->dxc && c.dyc == t->dyc) g = &c;
        if (!g) {
            e->sg.emplace_back();
            g = &e->sg.back();
            g->mx = t->mx;
            g->my = t->my;
            g->dxc = t->dxc;
            g->dyc = t->dyc;
        }
        g->members.push_back(i);
        EnsFineGroup* f = nullptr;
        for (auto& c : g->fine)
            if (c.lv == h->levels) f = &c;
        if (!f) {
            g->fine.emplace_back();
            f = &g->fine.back();
            f->lv = h->levels;
        }
        f->members.push_back(i);
        if (h->f2d) f->f2d = true;
    }
    // the groups with the most fine points first (their branches start first)
    auto points = [&](const EnsSolveGroup& g) {
        double p = 0;
        for (int i : g.members) p += (double)e->m[i]->nx * e->m[i]->ny;
        return p;
    };
    std::stable_sort(e->sg.begin(), e->sg.end(),
                     [&](const EnsSolveGroup& a, const EnsSolveGroup& b) { return points(a) > points(b); });
    for (auto& g : e->sg) {
        const std::vector<int> cands = batch_engines(e, g);
        g.engine = 0;
        if (cands.empty()) continue;
        const int nm = (int)g.members.size();
        std::vector<SolveMember<T>> tab(3 * (size_t)nm);
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < nm; ++j) {
                qg_ctx* h = e->m[g.members[j]];
                SolveMember<T>& M = tab[(size_t)k * nm + j];
                M = {};
                if (h->levels == 0) {
                    M.in[0] = static_cast<const T*>(h->w[k]);
                    M.nin = 1;
                    M.part_px = M.part_py = 1;
                    M.out = static_cast<T*>(h->psi);
                } else {
                    for (int q = 0; q < 4; ++q) M.in[q] = plane<T>(h->part, h->plane_c, q);
                    M.nin = 4;
                    M.part_px = fine_part_period_x(h->levels);
                    M.part_py = fine_part_period_y(h->levels, h->fine_rows);
                    M.out = static_cast<T*>(h->cpsi);
                }
                M.tr = static_cast<T*>(h->ct);
                M.work = static_cast<T*>(h->cw);
                M.err = h->derr;
            }
        const size_t nq = 2 + 3 * (size_t)nm;
        QG_TRY_E(ens_alloc(e, &g.dmem, tab.size() * sizeof(SolveMember<T>)));
        QG_TRY_E(ens_alloc(e, reinterpret_cast<void**>(&g.dq), nq * sizeof(unsigned)));
        if (cudaMemcpy(g.dmem, tab.data(), tab.size() * sizeof(SolveMember<T>),
                       cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(g.dq, 0, nq * sizeof(unsigned)) != cudaSuccess)
            return QG_ERR_CUDA;
        g.engine = cands[0];
    }
    const int TX = fine_block_cols();
    const int RC = ensemble_tile_rows(sizeof(T));
    for (auto& g : e->sg) {
        for (auto& f : g.fine) {
            const int nm = (int)f.members.size();
            std::vector<FineMember<T>> tab(3 * (size_t)nm);
            std::vector<int4> tiles;
            for (int j = 0; j < nm; ++j) {
                qg_ctx* h = e->m[f.members[j]];
                const LevelTables* t = nullptr;
                qg_status st = get_level(h, h->levels, &t);
                if (st != QG_OK) return st;
                for (int k = 0; k < 3; ++k) {
                    FineMember<T>& M = tab[(size_t)k * nm + j];
                    M.w = h->tm_halo[k][0];
                    M.wn = h->tm_int[0][0];
                    M.psi = h->tm_psi;
                    M.f = h->tm_f;
                    M.p = fused_params<T>(h, k, *t);
                }
                const int gx = (h->nx + TX - 1) / TX, gy = (h->ny + RC - 1) / RC;
                for (int by = 0; by < gy; ++by)
                    for (int bx = 0; bx < gx; ++bx) tiles.push_back(make_int4(j, bx, by, 0));
            }
            f.ntiles = (int)tiles.size();
            QG_TRY_E(ens_alloc(e, &f.dmem, tab.size() * sizeof(FineMember<T>)));
            QG_TRY_E(ens_alloc(e, reinterpret_cast<void**>(&f.dtiles), tiles.size() * sizeof(int4)));
            if (cudaMemcpy(f.dmem, tab.data(), tab.size() * sizeof(FineMember<T>),
                           cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(f.dtiles, tiles.data(), tiles.size() * sizeof(int4),
                           cudaMemcpyHostToDevice) != cudaSuccess)
                return QG_ERR_CUDA;
        }
    }
    // each group's solve engine, timed over whole group steps on the
    // members' buffers (which then return to rest) while the members hold
    // no user state, else over solves alone
    bool timed = false;
    for (auto& g : e->sg) {
        if (!g.engine) continue;
        bool t = false;
        QG_TRY_E(tune_group<T>(e, g, batch_engines(e, g), &t));
        timed = timed || t;
    }
    if (timed && e->fresh)
        for (qg_ctx* h : e->m) QG_TRY_E(rest_buffers(h, e->stream));
    return QG_OK;
}

// The batched solve of stage k of group g with engine `engine`.
template <typename T>
qg_status group_solve(qg_ensemble e, const EnsSolveGroup& g, int engine, int k, cudaStream_t s) {
    using C = typename Cx<T>::type;
    qg_ctx* h0 = e->m[g.members[0]];
    const LevelTables* t = nullptr;
    qg_status st = get_level(h0, h0->levels, &t);
    if (st != QG_OK) return st;
    SolveParams<T> P = {};
    P.mx = t->mx;
    P.my = t->my;
    P.layers = 1;
    P.ld = t->ldc;
    P.ld_tr = h0->ld_t;
    P.twx = static_cast<const C*>(t->twx);
    P.twy = static_cast<const C*>(t->twy);
    if (is_warp_engine(engine) || engine == kStreamEngine) {
        const int tab = engine == kStreamEngine ? 1 : engine - 32;   // engine 50: radix 16
        P.ptx = static_cast<const C*>(t->ptx[tab]);
        P.pty = static_cast<const C*>(t->pty[tab]);
    }
    P.lamx = static_cast<const T*>(t->lamx);
    P.lamy = static_cast<const T*>(t->lamy);
    P.scale = (T)((2.0 / t->mx) * (2.0 / t->my));
    P.bar = g.dq;
    P.err = h0->derr;
    P.batch = static_cast<const SolveMember<T>*>(g.dmem) + (size_t)k * g.members.size();
    P.nbatch = (int)g.members.size();
    P.no_pdl = kEnsemblePdl ? 0 : 1;
    if (engine == kMatrixEngine || engine == kTcEngine) {
        if constexpr (std::is_same<T, float>::value) {
            return cuda_status(h0, engine == kTcEngine
                                       ? launch_solve_tc(P, static_cast<const float*>(t->tctab), s)
                                       : launch_solve_mtx(P, static_cast<const float*>(t->mtab), s));
        } else {
            return QG_ERR_CUDA;
        }
    }
    return cuda_status(h0, launch_solve<T>(P, engine, s));
}

// One step of group g outside a graph, for timing: per stage the batched
// solve with `engine` and the batched fine stages.
template <typename T>
qg_status group_step_eager(qg_ensemble e, const EnsSolveGroup& g, int engine, cudaStream_t s) {
    for (int k = 0; k < 3; ++k) {
        QG_TRY_E(group_solve<T>(e, g, engine, k, s));
        for (const auto& f : g.fine) {
            const FineMember<T>* fm =
                static_cast<const FineMember<T>*>(f.dmem) + (size_t)k * f.members.size();
            if (launch_fine_batch<T>(fm, f.dtiles, f.ntiles, f.lv, f.f2d, kEnsemblePdl, s,
                                     ensemble_tile_rows(sizeof(T))) != cudaSuccess)
                return QG_ERR_CUDA;
        }
    }
    return QG_OK;
}

// The batched solve's engine for a group: each candidate timed, the fastest
// kept.  An ensemble being created times whole group steps (solves and fine
// stages on the members' own buffers: the solve alone ranks the engines
// differently, as for one basin) and *timed tells the caller to return the
// buffers to rest; a later rebuild, whose members hold state, times stage-1
// solves alone (they overwrite only work arrays and streamfunctions that
// every stage recomputes).  Results are cached per (grid, spacings,
// members, dtype) for the process and in the QG_TUNE_CACHE file; a cached
// engine that is no longer a candidate is timed again.

template <typename T>
qg_status tune_group(qg_ensemble e, EnsSolveGroup& g, const std::vector<int>& cands,
                     bool* timed) {
    *timed = false;
    if (cands.size() == 1) {
        g.engine = cands[0];
        return QG_OK;
    }
    const GroupKey key(g.mx, g.my, g.dxc, g.dyc, (int)g.members.size(), (int)sizeof(T));
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        tune_file_load();
    }
    {
        std::lock_guard<std::mutex> lock(g_batch_tune_mutex);
        auto it = g_batch_tune.find(key);
        if (it != g_batch_tune.end() &&
            std::find(cands.begin(), cands.end(), it->second) != cands.end()) {
            g.engine = it->second;
            return QG_OK;
        }
    }
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return QG_ERR_CUDA;
    *timed = true;
    float best = 1e30f;
    int pick = cands[0];
    for (int cand : cands) {
        bool ok = true;
        auto unit = [&]() {
            return (e->fresh ? group_step_eager<T>(e, g, cand, e->stream)
                             : group_solve<T>(e, g, cand, 0, e->stream)) == QG_OK;
        };
        for (int r = 0; r < 2 && ok; ++r) ok = unit();
        ok = ok && cudaEventRecord(a, e->stream) == cudaSuccess;
        for (int r = 0; r < 5 && ok; ++r) ok = unit();
        ok = ok && cudaEventRecord(b, e->stream) == cudaSuccess &&
             cudaEventSynchronize(b) == cudaSuccess;
        float ms = 1e30f;
        if (ok && cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms < best) {
            best = ms;
            pick = cand;
        }
        (void)cudaGetLastError();
        for (int i : g.members) e->m[i]->latched = QG_OK;   // a candidate failing is a result
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    g.engine = pick;
    std::lock_guard<std::mutex> lock(g_batch_tune_mutex);
    g_batch_tune[key] = pick;
    tune_file_store_group(key, pick);
    return QG_OK;
}

// Enqueue the three stages of one group's step on s (captured).
template <typename T>
qg_status group_enqueue(qg_ensemble e, const EnsSolveGroup& g, cudaStream_t s) {
    for (int k = 0; k < 3; ++k) {
        qg_ctx* h0 = e->m[g.members[0]];
        const LevelTables* t = nullptr;
        qg_status st = get_level(h0, h0->levels, &t);
        if (st != QG_OK) return st;
        if (!g.engine) {
            // the members' own solves
            for (int i : g.members) {
                qg_ctx* h = e->m[i];
                const LevelTables* ti = nullptr;
                st = get_level(h, h->levels, &ti);
                if (st != QG_OK) return st;
                h->kernels_per_step = 0;
                h->capturing = true;
                if (h->levels == 0)
                    st = solve_level<T>(h, *ti, h->w[k], h->ct, h->ld_t, h->plane_t, h->cw,
                                        h->psi, h->plane_f, s, 1);
                else
                    st = solve_level<T>(h, *ti, h->part, h->ct, h->ld_t, h->plane_t, h->cw,
                                        h->cpsi, h->plane_c, s, 4);
                h->capturing = false;
                e->kernels += h->kernels_per_step;
                if (st != QG_OK) return st;
            }
        } else {
            QG_TRY_E(group_solve<T>(e, g, g.engine, k, s));
            e->kernels += solve_launches(g.engine, g.mx, g.my, true);
        }
        if (k == 0) {
            for (int i : g.members) {
                qg_ctx* h = e->m[i];
                const bool fine = h->levels == 0;
                if (h->stats) {
                    QG_TRY_E(cuda_status(h, launch_accumulate<T>(
                        h->stat_acc, static_cast<const T*>(fine ? h->psi : h->cpsi),
                        (fine ? h->plane_f : h->plane_c) * h->layers, s)));
                    QG_TRY_E(cuda_status(h, launch_accumulate<T>(
                        h->stat_acc_w, static_cast<const T*>(h->w[0]), h->plane_f * h->layers, s)));
                    e->kernels += 2;
                }
                if (h->cfl > 0.0) {
                    const LevelTables* ti = nullptr;
                    st = get_level(h, h->levels, &ti);
                    if (st != QG_OK) return st;
                    QG_TRY_E(cuda_status(h, cudaMemsetAsync(h->dclock, 0, sizeof(double), s)));
                    QG_TRY_E(cuda_status(h, launch_cfl_max<T>(
                        static_cast<const T*>(fine ? h->psi : h->cpsi), fine ? h->ldf : ti->ldc,
                        h->nx, h->ny, h->levels, h->dx, h->dy,
                        reinterpret_cast<unsigned long long*>(h->dclock), s)));
                    ++e->kernels;
                }
            }
        }
        for (const auto& f : g.fine) {
            const FineMember<T>* fm =
                static_cast<const FineMember<T>*>(f.dmem) + (size_t)k * f.members.size();
            QG_TRY_E(cuda_status(e->m[f.members[0]],
                                 launch_fine_batch<T>(fm, f.dtiles, f.ntiles, f.lv, f.f2d,
                                                      kEnsemblePdl, s,
                                                      ensemble_tile_rows(sizeof(T)))));
            ++e->kernels;
        }
    }
    return QG_OK;
}

// Enqueue one ensemble step on s (captured into the graph): the groups'
// chains on branches forked from and joined back into s.
template <typename T>
qg_status ensemble_enqueue(qg_ensemble e, cudaStream_t s) {
    e->kernels = 0;
    QG_TRY_E(ensemble_lanes(e, e->sg.size()));
    if (cudaEventRecord(e->ev[0], s) != cudaSuccess) return QG_ERR_CUDA;
    for (size_t k = 0; k < e->sg.size(); ++k) {
        if (cudaStreamWaitEvent(e->lanes[k], e->ev[0], 0) != cudaSuccess) return QG_ERR_CUDA;
        QG_TRY_E(group_enqueue<T>(e, e->sg[k], e->lanes[k]));
        if (cudaEventRecord(e->ev[1 + k], e->lanes[k]) != cudaSuccess ||
            cudaStreamWaitEvent(s, e->ev[1 + k], 0) != cudaSuccess)
            return QG_ERR_CUDA;
    }
    return QG_OK;
}

qg_status ensemble_build(qg_ensemble e) {
    // a member whose own step changed (new forcing field, adaptive step,
    // statistics, solver, fault switch) invalidates the ensemble's graph
    bool stale = e->gen.size() != e->m.size();
    for (size_t i = 0; i < e->m.size() && !stale; ++i) stale = e->gen[i] != e->m[i]->graph_gen;
    if (e->gexec && !stale) return QG_OK;
    cudaStreamSynchronize(e->stream);
    if (e->gexec) {
        cudaGraphExecDestroy(e->gexec);
        e->gexec = nullptr;
    }
    if (e->graph) {
        cudaGraphDestroy(e->graph);
        e->graph = nullptr;
    }
    const bool f64 = e->m[0]->dtype == QG_F64;
    qg_status st = f64 ? ensemble_tables<double>(e) : ensemble_tables<float>(e);
    if (st != QG_OK) return st;
    if (cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return QG_ERR_CUDA;
    st = f64 ? ensemble_enqueue<double>(e, e->cap) : ensemble_enqueue<float>(e, e->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(e->cap, &g);
    if (st != QG_OK || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        return st != QG_OK ? st : QG_ERR_CUDA;
    }
    e->graph = g;
    if (cudaGraphInstantiate(&e->gexec, g, 0) != cudaSuccess) {
        (void)cudaGetLastError();
        return QG_ERR_CUDA;
    }
    e->gen.clear();
    for (qg_ctx* h : e->m) e->gen.push_back(h->graph_gen);
    return QG_OK;
}

}  // namespace

extern "C" {

qg_status qg_ensemble_create(const qg_basin* basins, const double* Re, const double* Ro,
                             const int* levels, int count, qg_dtype dtype,
                             void* cuda_stream, qg_ensemble* out) {
    if (!basins || !Re || !Ro || !levels || !out || count < 1 || count > 4096) return QG_ERR_ARG;
    *out = nullptr;
    qg_ensemble e = new (std::nothrow) qg_ensemble_s();
    if (!e) return QG_ERR_OOM;
    e->stream = static_cast<cudaStream_t>(cuda_stream);
    for (int i = 0; i < count; ++i) {
        qg_handle h = nullptr;
        const qg_status s = create_ctx(&basins[i], 1, Re[i], Ro[i], 0.0, levels[i], dtype,
                                       cuda_stream, true, &h);
        if (s != QG_OK) {
            ensemble_free(e);
            return s;
        }
        e->m.push_back(h);
    }
    const bool ok = cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        ensemble_free(e);
        (void)cudaGetLastError();
        return QG_ERR_CUDA;
    }
    // the graph is built now, while the members' buffers may run timing steps
    e->fresh = true;
    const qg_status s = ensemble_build(e);
    e->fresh = false;
    if (s != QG_OK) {
        ensemble_free(e);
        (void)cudaGetLastError();
        return s;
    }
    *out = e;
    return QG_OK;
}

qg_status qg_ensemble_member(qg_ensemble e, int index, qg_handle* out) {
    if (!e || !out || index < 0 || index >= (int)e->m.size()) return QG_ERR_ARG;
    *out = e->m[index];
    return QG_OK;
}

qg_status qg_ensemble_step(qg_ensemble e, int64_t n) {
    NvtxRange nvtx_range("qg_ensemble_step");
    if (!e || n < 0) return QG_ERR_ARG;
    for (qg_ctx* h : e->m)
        if (h->latched != QG_OK) return qg_last_error(h);
    if (n == 0) return QG_OK;
    // the members' partial sums of R^l w^n are made on the ensemble stream
    for (qg_ctx* h : e->m) {
        if (h->part && !h->part_valid) {
            const qg_status s = h->dtype == QG_F64 ? init_partials<double>(h, h->stream)
                                                   : init_partials<float>(h, h->stream);
            if (s != QG_OK) return s;
            h->part_valid = true;
        }
    }
    qg_status s = ensemble_build(e);
    if (s != QG_OK) return s;
    for (qg_ctx* h : e->m)
        if (h->stats) h->stat_count += n;
    for (int64_t k = 0; k < n; ++k)
        if (cudaGraphLaunch(e->gexec, e->stream) != cudaSuccess) {
            (void)cudaGetLastError();
            return QG_ERR_CUDA;
        }
    return QG_OK;
}

qg_status qg_ensemble_kernel_count(qg_ensemble e, int64_t* count) {
    if (!e || !count) return QG_ERR_ARG;
    const qg_status s = ensemble_build(e);
    if (s != QG_OK) return s;
    *count = e->kernels;
    return QG_OK;
}

qg_status qg_ensemble_synchronize(qg_ensemble e) {
    if (!e) return QG_ERR_ARG;
    if (cudaStreamSynchronize(e->stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return QG_ERR_CUDA;
    }
    qg_status first = QG_OK;
    for (qg_ctx* h : e->m) {
        const qg_status s = qg_synchronize(h);
        if (first == QG_OK) first = s;
    }
    return first;
}

qg_status qg_ensemble_destroy(qg_ensemble e) {
    ensemble_free(e);
    return QG_OK;
}

}  // extern "C"
