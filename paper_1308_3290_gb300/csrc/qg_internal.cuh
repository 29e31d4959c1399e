// Internal declarations shared by the CUDA translation units of libqgcgp.
//
// Device layout of every grid of a basin ("padded node layout"): a level with
// n_x x n_y intervals is stored as n_y + 1 rows of `ld` elements, node (i, j)
// at [j * ld + i], i = 0..n_x, j = 0..n_y; ld = round_up(n_x + 1, 32).  The
// wall nodes (i = 0, n_x and j = 0, n_y) always hold 0 and the columns past
// n_x are never read.  Row j, entries 0..n_x-1, is exactly the length-n_x
// input f_0..f_{n_x-1} (f_0 = 0) of the DST-I engine, so the solver runs on
// the stored rows without repacking.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qg.h"

namespace qg {

template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }
inline int ilog2(int v) { int r = 0; while ((1 << r) < v) ++r; return r; }
inline bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Shape of one DST launch: NB butterflies per thread and pass, `lanes`
// independent sequences per CTA.
struct DstLaunch {
    int nb;
    int lanes;
};

// ---- kernels (declared here, defined in dst.cu / stencil.cu / diag.cu) ----

// The elliptic solve of one level (solve.cu): x pass of `in` (the sum of
// nin planes per layer; with nin == 4 plane 1 is read only at columns
// k % part_px == 0, plane 2 at rows r % part_py == 0, plane 3 at both;
// part_px and part_py are powers of two, tested with masks), the
// y pass with the eigenvalue division (one layer: lap_h psi = rhs) or the
// coupled solve of Eqs. isub-1/2 (two layers), the inverse x pass into
// `out`.  in / work / out have the level's padded layout (pitch ld), tr the
// transposed layout (mx + 1 rows of pitch ld_tr).  bar: two zero-initialised
// counters of the grid barrier.  One cooperative launch, or (split) one
// plain launch per pass.
// Per-member fields of a batched solve launch (ensembles): the members of a
// batch share the elliptic grid and its tables (mx, my, ld, ld_tr, twiddle
// and eigenvalue tables, scale); each has its own right-hand side planes,
// transposed spectrum, work and output arrays and error flag.  One layer.
template <typename T>
struct SolveMember {
    const T* in[4];
    int nin, part_px, part_py;
    T* tr;
    T* work;
    T* out;
    int* err;
};

template <typename T>
struct SolveParams {
    int mx, my, layers;
    const T* in[2][4];
    int nin, part_px, part_py;
    int ld;
    T* tr[2];
    int ld_tr;
    T* work[2];
    T* out[2];
    const typename Cx<T>::type* twx;   // e^{i pi t/mx}, t < 2 mx
    const typename Cx<T>::type* twy;   // e^{i pi t/my}, t < 2 my
    const typename Cx<T>::type* ptx;   // warp-group engine: per-pass twiddles for
    const typename Cx<T>::type* pty;   //   2 mx and 2 my (see pass_table_size)
    const T* lamx;                      // (2 cos(pi k/mx) - 2)/dx^2, k = 0..mx
    const T* lamy;                      // (2 cos(pi l/my) - 2)/dy^2, l = 0..my
    T scale, Ro, f1, f2;
    unsigned* bar;
    unsigned bar_extra;  // arrivals the grid barrier waits for beyond the grid
                         // (0; 1 only under fault injection: never released)
    int* err;
    int split;           // 0: the three passes in one cooperative launch with
                         // grid barriers; 1: three plain launches, one per pass
    int phase;           // the pass a split launch runs (set by launch_solve)
    // Batch (ensembles): when non-null, one launch solves the nbatch
    // members' systems; their fields replace in/nin/part_*/tr/work/out/err
    // of this struct (split must be 0).  Warp-group engines: a work queue
    // whose counters are bar[0 .. 2 + 3 nbatch), zero before the first
    // launch and left zero by every launch; the matrix form: one CTA per
    // member.
    const SolveMember<T>* batch;
    int nbatch;
    int no_pdl;          // 1: launch without programmatic dependent launch
                         // (kernels on concurrent branches: a dependent that
                         // started early would hold SM resources idle)
};
// engine: base radix of the FFT passes of the shared-memory engine, 4 or 16
// (see dst_engine.cuh), or the warp-group engine of solve32.cu with 32, 16
// or 8 values per thread (engines 32, 33, 34)
template <typename T>
cudaError_t launch_solve(const SolveParams<T>& P, int engine, cudaStream_t s);
size_t solve_smem_bytes(int mx, int my, size_t esz, int engine);
bool solve_engine_supports(int mx, int my, size_t esz, int engine);
// The warp-group engine's twiddle table for an FFT of length L = 2N with
// `rad` values per thread: for each pass p >= 1 (radix R_p, sub-transform
// size Ns_p), R_p x Ns_p entries e^{-2 pi i r k / (R_p Ns_p)} at
// [r Ns_p + k], passes in order.
size_t pass_table_size(int L, int rad);
void pass_table(int L, int rad, double* re, double* im);   // pass_table_size entries
template <typename T>
cudaError_t launch_solve32(const SolveParams<T>& P, int rad, cudaStream_t s);
size_t solve32_smem_bytes(int mx, int my, size_t esz, int rad);
bool solve32_supports(int mx, int my, int rad, size_t esz);
// engines 32, 33, 34: the warp-group engine with 32, 16, 8 values per thread
inline int warp_engine_radix(int engine) { return engine == 34 ? 8 : (engine == 33 ? 16 : 32); }
inline bool is_warp_engine(int engine) { return engine >= 32 && engine <= 34; }
// engine 50: one CTA per sequence pair, three launches, radix-16 passes
// with the values in registers (solve_stream.cu); it takes the radix-16
// pass tables of engine 33 (ptx/pty)
constexpr int kStreamEngine = 50;
bool stream_supports(int mx, int my, size_t esz);
template <typename T>
cudaError_t launch_solve_stream(const SolveParams<T>& P, cudaStream_t s);
// batched engine-50 solves that run as one work-queue launch
bool stream_queue_ok(int mx, int my, int layers);
// the kernels one solve of an engine launches (a batch of members: `batch`)
inline int solve_launches(int engine, int mx = 0, int my = 0, bool batch = false) {
    if (engine != kStreamEngine) return 1;
    return batch && stream_queue_ok(mx, my, 1) ? 1 : 3;
}

// Full-weighting restriction applied `levels` times, as one hat-weighted
// sum (fine -> level `levels`), interior coarse nodes only.
template <typename T>
cudaError_t launch_restrict(const T* fine, int ldf, T* coarse, int ldc,
                            int mx, int my, int levels, cudaStream_t s);

// Bilinear prolongation applied `levels` times (level `levels` -> fine),
// interior fine nodes only.
template <typename T>
cudaError_t launch_prolong(const T* coarse, int ldc, T* fine, int ldf,
                           int nx, int ny, int levels, cudaStream_t s);

// Constants of one fine-grid stage of the one-layer model.
template <typename T>
struct StageParams {
    int nx, ny, ld;
    T c_jac;      // 1 / (12 dx dy): Arakawa (J1 + J2 + J3) / 3 / (4 dx dy)
    T c_beta;     // 1 / (12 Ro dx): closed form of (1/Ro) J(psi, y)
    T c_lapx;     // 1 / (Re dx^2)
    T c_lapy;     // 1 / (Re dy^2)
    T dt;
    T a;          // weight of w^n in the TVDRK3 combination
    T b;          // weight of (w^(s) + dt G)
};

// One TVDRK3 stage on the fine grid: w_out = a w_n + b (w + dt G(psi, w)),
// G = -J(psi, w) - (1/Ro) J(psi, y) + (1/Re) lap w + F.  F is the per-row
// forcing `frow` (length ny + 1), or the padded field `f2d` when non-null.
template <typename T>
cudaError_t launch_fine_stage(const T* psi, const T* w, const T* wn, T* wout,
                              const T* frow, const T* f2d,
                              const StageParams<T>& p, cudaStream_t s);

// Adjoint kernels (adjoint.cu) of the one-layer step.
template <typename T>
struct AdjParams {
    int nx, ny, ld;
    T c_jac, c_beta;      // 1/(12 dx dy), 1/(12 Ro dx)
    T c_lapx, c_lapy;     // 1/(Re dx^2), 1/(Re dy^2)
    T dt, a, b;           // time step and the stage's TVDRK3 weights
    T inv_dx2, inv_dy2, dxdy;
};
// out = J(w, lam) - (1/Ro) J(lam, y)
template <typename T>
cudaError_t launch_adj_source(const T* w, const T* lam, T* out, const AdjParams<T>& p,
                              cudaStream_t s);
// next = [next +] b lam + b dt (J(psi, lam) + (1/Re) lap lam - phi);
// acc += a lam; g += b dt lam
template <typename T>
cudaError_t launch_adj_stage(const T* psi, const T* lam, const T* phi, T* next, T* acc, T* g,
                             const AdjParams<T>& p, bool accumulate, cudaStream_t s);
// out = -dx dy lap psi
template <typename T>
cudaError_t launch_energy_source(const T* psi, T* out, const AdjParams<T>& p, cudaStream_t s);
// dense (exchange layout) += scale * padded (interior)
template <typename T>
cudaError_t launch_add_to_dense(T* dense, const T* padded, double scale, int nx, int ny, int ld,
                                cudaStream_t s);

// Fused one-layer stage (fused.cu): prolongation of psi on load, the stage
// update, and restriction of the result into four partial-sum planes.
template <typename T>
struct FusedParams {
    int nx, ny, ld;        // fine grid intervals and pitch
    const T* psi;          // l = 0: fine psi; l >= 1: elliptic-grid psi
    int ldp;               // pitch of psi
    const T* w;            // w^(s)
    const T* wn;           // w^n (read only when a != 0; may alias wout)
    T* wout;               // w^(s+1)
    const T* frow;         // forcing per fine row
    const T* f2d;          // forcing field or null
    T* part[4];            // restriction partial planes (l >= 1)
    int ldc;               // their pitch
    int* err;              // set to 1 when a bounded wait runs out
    T c_jac, c_beta, c_lapx, c_lapy, dt, a, b;
    // Adaptive step (Eq. dt): when umax is non-null, dt = min(dt_cap,
    // cfl_h / u) with u the double whose bits *umax holds (u = 0: dt_cap).
    const unsigned long long* umax;
    double cfl_h, dt_cap;
    double* clock;         // {time, last dt}: the last stage adds its dt
    int last_stage;
    // Two-layer stage (Section 2.2, Eq. ge-non; layer i, other layer j): the
    // state is Q_i, the dissipation acts on w_i = Q_i/Ro + k_p (psi_i - psi_j)
    // (Eq. pv-non, k_p = Fr/(delta_i Ro)), c_beta = 1/(12 dx), c_lap = A/dx^2,
    // A/dy^2, drag = sigma for the bottom layer; frow may be null (no wind).
    const T* psi_o;        // the other layer's elliptic-grid psi (two layers)
    T inv_Ro, k_p, drag;
};

// acc[e] += src[e] for the n elements of a padded plane (FP64 sums).
template <typename T>
cudaError_t launch_accumulate(double* acc, const T* src, size_t n, cudaStream_t s);
// dense[(j-1)(nx-1) + i-1] = scale * (acc prolonged `levels` times)(i, j)
template <typename T>
cudaError_t launch_mean_out(T* dense, const double* acc, int ldacc, double scale, int nx,
                            int ny, int levels, cudaStream_t s);

// dense[(j-1)(nx-1) + i-1] = scale * acc[j ld + i] + y0 + j dy (fine grid):
// the time-mean potential vorticity from a sum of states
template <typename T>
cudaError_t launch_mean_q_out(T* dense, const double* acc, int ld, double scale, int nx, int ny,
                              double y0, double dy, cudaStream_t s);

// u = max over interior fine nodes of |psi_x| and |psi_y| (central
// differences, Eq. dt) of psi prolonged `levels` times from `psi` (pitch
// ldp); atomically max-ed into *umax as the bits of a non-negative double.
template <typename T>
cudaError_t launch_cfl_max(const T* psi, int ldp, int nx, int ny, int levels, double dx,
                           double dy, unsigned long long* umax, cudaStream_t s);

// TMA tensor maps of the inputs of one fused launch: w^(s) and the fine psi
// with halo boxes, w^n and the forcing field with interior boxes.  Unused
// maps may hold anything (they are not dereferenced).
struct FineMaps {
    CUtensorMap w, wn, psi, f;
};
// rows: the fine rows per CTA and ry the fine rows each thread sweeps
// (fine_tile_rows and fine_rows_per_thread, or a tuned pair that
// fine_rows_supported accepts; the tensor maps' boxes must match rows)
template <typename T>
cudaError_t launch_fine_fused(const FusedParams<T>& p, const FineMaps& m, int levels,
                              cudaStream_t s, bool two_layer, int rows, int ry);
// One member of a batched fine-stage launch (ensembles): the tensor maps of
// its stage and its parameters, in device memory (the TMA unit reads the
// maps from there; 64-byte aligned).
template <typename T>
struct alignas(64) FineMember {
    CUtensorMap w, wn, psi, f;
    FusedParams<T> p;
};
// One layer: CTA c sweeps the tile (tiles[c].y, tiles[c].z) of member
// tiles[c].x; `levels` is every member's CGP level; forcing_field when any
// member uses a forcing field; tiles of `rows` fine rows
// (ensemble_tile_rows).
template <typename T>
cudaError_t launch_fine_batch(const FineMember<T>* fm, const int4* tiles, int ntiles, int levels,
                              bool forcing_field, bool pdl, cudaStream_t s, int rows);
size_t fine_tile_rows(size_t esz);   // default fine rows per CTA
int ensemble_tile_rows(size_t esz);  // fine rows per CTA of ensemble members
int fine_rows_per_thread(int levels);   // default rows a thread sweeps
bool fine_rows_supported(size_t esz, int layers, int levels, int rows, int ry);  // tuned pairs
int fine_part_period_x(int levels);  // coarse columns between tile edges
int fine_part_period_y(int levels, int rows);  // coarse rows between CTA edges
int fine_halo_cols();                // columns of a halo box
int fine_block_cols();               // columns of an interior box

// 2-D tensor map over a padded level array (x = 0..n_x, y = 0..n_y), box
// bw x bh, zero fill outside.
cudaError_t make_tensor_map(CUtensorMap* m, const void* base, int nx, int ny, int ld,
                            size_t esz, int bw, int bh);

// Two-layer stage (Eq. ge-non): both layers in one pass.
template <typename T>
struct StageParams2 {
    int nx, ny, ld;
    T c_jac, c_beta;     // 1/(12 dx dy), 1/(12 dx)
    T inv_Ro;            // 1/Ro
    T f1, f2;            // Fr/delta, Fr/(1-delta)
    T A_dx2, A_dy2;      // A/dx^2, A/dy^2
    T sigma;
    T dt, a, b;
};
template <typename T>
cudaError_t launch_fine_stage2(const T* psi1, const T* psi2, const T* q1,
                               const T* q2, const T* qn1, const T* qn2,
                               T* out1, T* out2, const T* frow,
                               const StageParams2<T>& p, cudaStream_t s);

// Deterministic FP64 diagnostics: per-CTA partial sums of the squared edge
// differences of psi along x and y, of w^2, and per-CTA maxima of |psi_x|,
// |psi_y|; then one CTA folds them in a fixed order into out[0..3].
template <typename T>
cudaError_t launch_diagnostics(const T* psi, const T* w, int nx, int ny, int ld,
                               double dx, double dy, double* partial,
                               int nblocks, double* out, cudaStream_t s);
int diag_blocks();
// acc[0] += c0 out[0] + c1 out[1] (out: the FP64 results of launch_diagnostics)
cudaError_t launch_energy_add(const double* out, double c0, double c1, double* acc,
                              cudaStream_t s);

// ---- geometric multigrid (multigrid.cu) ----------------------------------
constexpr int kMaxTail = 14;          // levels the one-CTA tail can hold
template <typename T>
struct MGLevelDesc {                  // one grid of the hierarchy
    T* psi;                           // (my+1) rows of pitch ld, zero walls
    const T* rhs;                     // right-hand side, pitch ldr
    T* rhs_w;                         // the same, writable (levels >= 1)
    int mx, my, ld, ldr;
    T cx, cy;                         // 1/dx^2, 1/dy^2 of this grid
};
template <typename T>
struct MGTail {                       // levels handled by one CTA in shared memory
    int n;
    int mx[kMaxTail], my[kMaxTail];
    T cx[kMaxTail], cy[kMaxTail];
    T* psi;                           // first tail level (global): guess in, result out
    const T* rhs;
    int ld, ldr;
};
template <typename T>
struct MGSumParams {                  // rhs = in[0] + in[1] + ..., psi = 0 if zero
    const T* in[4];
    int nin, ld_in;
    T* rhs;
    T* psi;
    int mx, my, ld, zero;
};
size_t mg_tail_smem(const int* mx, const int* my, int n, size_t esz);
int mg_cycle_launches(int tail);      // kernels of one V-cycle
cudaError_t mg_reserve_tail_smem(size_t bytes, size_t esz);
template <typename T>
cudaError_t launch_mg_sum(const MGSumParams<T>& q, cudaStream_t s);
template <typename T>
cudaError_t launch_mg_cycle(const MGLevelDesc<T>* lv, int nl, int tail, cudaStream_t s);

// Resident CTAs per SM and SM count for `kernel` at (threads, smem) on the
// current device, its dynamic shared-memory limit raised to smem; looked up
// once per (kernel, threads, smem, device) and cached (the eager launch
// paths -- adjoint sweeps, stand-alone solves -- launch thousands of times).
cudaError_t launch_shape(const void* kernel, int threads, size_t smem, int* per_sm, int* nsm);

// Bounds-checked builds (bounds.cuh): the site of the first failed index
// check in each translation unit since the last query (0: none; always 0
// in normal builds), cleared by the query.
int bounds_site_fused();
int bounds_site_solve32();
int bounds_site_stencil();
int bounds_site_mtx();
int bounds_site_stream();

// Copies between the dense exchange layout and the padded node layout.
cudaError_t copy_in(void* padded, int ld, const void* dense, int nxm1,
                    int nym1, size_t esz, cudaStream_t s);
cudaError_t copy_out(void* dense, const void* padded, int ld, int nxm1,
                     int nym1, size_t esz, cudaStream_t s);

}  // namespace qg
