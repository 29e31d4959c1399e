// qg_poisson_solve_noalloc: the sine-transform Poisson solve without any
// device allocation.
//
// Some callers cannot call cudaMalloc: a host application that hands out all
// device memory through its own pool or a hard per-tenant quota, or a
// latency-critical loop in which cudaMalloc/cudaFree would synchronise the
// device and stall unrelated streams.  For them this entry point keeps its
// workspace (the padded work grid, its transposed spectrum, and the twiddle
// and eigenvalue tables) in
// one file-scope __device__ array of fixed size, kNoAllocBytes.  Every GPU
// that loads the library holds that array until the process exits.
//
// The array's name in host code is only a host-side stand-in, not a device
// address, so the first call on each device looks up the real address with
// cudaGetSymbolAddress while that device is current, and later calls reuse
// it.  Make that first call on a device before any stream capture begins.
// All calls share the one array and it keeps the contents of the last call:
// each call clears the part that must start at zero, and two calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on
// it.  Each call waits for its stream at the end and reads the solve's error
// word back (into a stack variable: no pinned buffer is allocated), so that a
// grid-barrier wait that ran out of its bound is reported as QG_ERR_TIMEOUT
// rather than as success.  The paper has no counterpart to this entry point.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "qg_internal.cuh"

namespace qg {
namespace {

constexpr size_t kNoAllocBytes = 32u << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Twiddle tables e^{i pi t/N} (t < 2N) of both directions and the 1-D
// eigenvalues of the 5-point Laplacian, computed in FP64 on the device and
// stored in the working precision.
template <typename T>
__global__ void noalloc_tables(typename Cx<T>::type* twx, int mx,
                               typename Cx<T>::type* twy, int my, T* lamx,
                               T* lamy, double dx, double dy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 2 * mx) {
        double s, c;
        sincospi((double)i / mx, &s, &c);
        twx[i].x = (T)c;
        twx[i].y = (T)s;
    }
    if (i < 2 * my) {
        double s, c;
        sincospi((double)i / my, &s, &c);
        twy[i].x = (T)c;
        twy[i].y = (T)s;
    }
    if (i <= mx) lamx[i] = (i == 0 || i == mx) ? T(0) : (T)((2.0 * cospi((double)i / mx) - 2.0) / (dx * dx));
    if (i <= my) lamy[i] = (i == 0 || i == my) ? T(0) : (T)((2.0 * cospi((double)i / my) - 2.0) / (dy * dy));
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Byte layout of the scratch for one request: padded grid, then the tables.
struct Layout {
    size_t grid, tr, twx, twy, lamx, lamy, bar, total;
};

Layout layout(int nx, int ny, size_t esz) {
    Layout L;
    const int ld = round_up(nx + 1, 32);
    const int ldt = round_up(ny + 1, 32);
    L.grid = 0;
    L.tr = align256((size_t)(ny + 1) * ld * esz);
    L.twx = L.tr + align256((size_t)(nx + 1) * ldt * esz);
    L.twy = L.twx + align256((size_t)4 * nx * esz);
    L.lamx = L.twy + align256((size_t)4 * ny * esz);
    L.lamy = L.lamx + align256((size_t)(nx + 1) * esz);
    L.bar = L.lamy + align256((size_t)(ny + 1) * esz);   // 2 barrier counters + error word
    L.total = L.bar + 256;
    return L;
}

template <typename T>
qg_status solve(unsigned char* base, const Layout& Lo, int nx, int ny, double dx,
                double dy, const void* rhs, void* psi, int engine, bool stall,
                cudaStream_t s) {
    using C = typename Cx<T>::type;
    const int ld = round_up(nx + 1, 32);
    T* grid = reinterpret_cast<T*>(base + Lo.grid);
    C* twx = reinterpret_cast<C*>(base + Lo.twx);
    C* twy = reinterpret_cast<C*>(base + Lo.twy);
    T* lamx = reinterpret_cast<T*>(base + Lo.lamx);
    T* lamy = reinterpret_cast<T*>(base + Lo.lamy);
    const size_t esz = sizeof(T);
    // the walls of the padded grid must be zero: clear the whole grid
    if (cudaMemsetAsync(grid, 0, (size_t)(ny + 1) * ld * esz, s) != cudaSuccess) return QG_ERR_CUDA;
    const int n = 2 * (nx > ny ? nx : ny) + 1;
    noalloc_tables<T><<<(n + 255) / 256, 256, 0, s>>>(twx, nx, twy, ny, lamx, lamy, dx, dy);
    if (cudaGetLastError() != cudaSuccess) return QG_ERR_CUDA;
    if (copy_in(grid, ld, rhs, nx - 1, ny - 1, esz, s) != cudaSuccess) return QG_ERR_CUDA;
    unsigned* bar = reinterpret_cast<unsigned*>(base + Lo.bar);
    if (cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), s) != cudaSuccess) return QG_ERR_CUDA;
    SolveParams<T> P = {};
    P.mx = nx;
    P.my = ny;
    P.layers = 1;
    P.in[0][0] = grid;
    P.nin = 1;
    P.part_px = P.part_py = 1;
    P.ld = ld;
    P.tr[0] = reinterpret_cast<T*>(base + Lo.tr);
    P.ld_tr = round_up(ny + 1, 32);
    P.work[0] = grid;
    P.out[0] = grid;
    P.twx = twx;
    P.twy = twy;
    P.lamx = lamx;
    P.lamy = lamy;
    P.scale = (T)((2.0 / nx) * (2.0 / ny));
    P.bar = bar;
    P.err = reinterpret_cast<int*>(bar + 2);
    P.bar_extra = stall ? 1u : 0u;
    if (launch_solve<T>(P, engine, s) != cudaSuccess) return QG_ERR_CUDA;
    int err = 0;
    if (cudaMemcpyAsync(&err, P.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return QG_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return QG_ERR_CUDA;
    if (err) return QG_ERR_TIMEOUT;
    // psi is written only when the solve completed
    if (copy_out(psi, grid, ld, nx - 1, ny - 1, esz, s) != cudaSuccess) return QG_ERR_CUDA;
    return QG_OK;
}

// The shared-memory FFT engine for an nx x ny request: base radix 16 for
// grids of 2^21 nodes or more, radix 4 below (the faster of the two there),
// falling back to the other radix when the first cannot take the grid's
// longer side or shared memory; 0 when neither can.
int pick_engine(int nx, int ny, size_t esz) {
    const int first = (long)nx * ny >= (1L << 21) ? 16 : 4;
    const int second = first == 16 ? 4 : 16;
    if (solve_engine_supports(nx, ny, esz, first)) return first;
    if (solve_engine_supports(nx, ny, esz, second)) return second;
    return 0;
}

}  // namespace
}  // namespace qg

using namespace qg;

extern "C" qg_status qg_poisson_solve_noalloc(int32_t nx, int32_t ny, double dx,
                                              double dy, qg_dtype dtype,
                                              const void* rhs, void* psi,
                                              void* cuda_stream) {
    if (!rhs || !psi) return QG_ERR_ARG;
    if (dtype != QG_F32 && dtype != QG_F64) return QG_ERR_ARG;
    if (!(dx > 0) || !(dy > 0)) return QG_ERR_ARG;
    if (!is_pow2(nx) || !is_pow2(ny) || nx < 8 || ny < 8 || nx > 8192 || ny > 8192)
        return QG_ERR_SHAPE;
    const size_t esz = dtype == QG_F64 ? 8 : 4;
    if (layout(nx, ny, esz).total > kNoAllocBytes) return QG_ERR_SHAPE;
    const int engine = pick_engine(nx, ny, esz);
    if (!engine) return QG_ERR_SHAPE;
    // QG_NOALLOC_STALL=1 (a test hook for the timeout path): the solve's first
    // grid barrier waits for one arrival more than the grid has, so its
    // bounded wait runs out and the call returns QG_ERR_TIMEOUT.
    const char* st = std::getenv("QG_NOALLOC_STALL");
    const bool stall = st && std::strcmp(st, "1") == 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return QG_ERR_NO_DEVICE;
    }
    if (dev < 0 || dev >= kMaxDevices) return QG_ERR_UNSUPPORTED;
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                (void)cudaGetLastError();
                return QG_ERR_CUDA;
            }
            g_scratch_addr[dev] = p;
        }
        base = static_cast<unsigned char*>(g_scratch_addr[dev]);
    }
    const Layout Lo = layout(nx, ny, esz);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    return dtype == QG_F64 ? solve<double>(base, Lo, nx, ny, dx, dy, rhs, psi, engine, stall, s)
                           : solve<float>(base, Lo, nx, ny, dx, dy, rhs, psi, engine, stall, s);
}
