/*
 * qg.h -- C ABI of the GB300-native coarse grid projection (CGP) time step
 * for quasigeostrophic ocean basins (San & Staples, "An Efficient Coarse Grid
 * Projection Method for Quasigeostrophic Models of Large-Scale Ocean
 * Circulation", arXiv 1308.3290).
 *
 * Every call returns a qg_status.  No C++ exception crosses this boundary.
 * Outputs are written only when the call returns QG_OK.  Work is enqueued on
 * the CUDA stream given to qg_create and runs asynchronously unless a call
 * says it synchronises; an error raised by such work is latched in the handle
 * and returned by the next call (and by qg_last_error).
 *
 * Grids.  A basin has nx x ny grid INTERVALS (Section 4.3 of the paper sums
 * over i = 1..N_x-1): nodes i = 0..nx, j = 0..ny, walls at the first and last
 * node of each direction, unknowns at the interior nodes.  Level l of a basin
 * is the grid with nx/2^l x ny/2^l intervals (Section 3, M = 2^-l N); level 0
 * is the fine grid, level `coarsening_levels` the elliptic (coarse) grid.
 *
 * Exchange layout.  Every field passed through this ABI is the interior of a
 * level-l grid as a dense row-major array of (ny_l - 1) rows of (nx_l - 1)
 * values, x fastest, in the handle's dtype (float for QG_F32, double for
 * QG_F64).  Pointers may be device pointers or host pointers (pageable host
 * memory makes the copy synchronous; pinned host memory keeps it
 * asynchronous: a kernel reads or writes it in place).  The caller owns every pointer it passes; the handle owns
 * its internal state and workspace (device memory allocated in qg_create).
 *
 * Threading.  One handle is used by one host thread at a time; calls on
 * distinct handles are independent.
 */
#ifndef QG_H
#define QG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum qg_status {
    QG_OK = 0,
    QG_ERR_ARG = 1,          /* NULL pointer, out-of-range scalar or level   */
    QG_ERR_SHAPE = 2,        /* grid not a power of two, or too small/large  */
    QG_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed  */
    QG_ERR_OOM = 4,          /* device allocation failed                     */
    QG_ERR_NONFINITE = 5,    /* the state holds NaN or Inf                   */
    QG_ERR_CFL = 6,          /* qg_set_cfl asked for a Courant number above
                                1, beyond what Eq. dt allows                */
    QG_ERR_TIMEOUT = 7,      /* a bounded device-side wait ran out           */
    QG_ERR_UNSUPPORTED = 8,  /* valid request the library does not provide   */
    QG_ERR_NO_DEVICE = 9     /* no usable CUDA device                        */
} qg_status;

typedef enum qg_dtype {
    QG_F32 = 0,  /* FP32 fields; FP64-generated twiddle/eigenvalue tables and
                    FP64 energy/enstrophy reductions                         */
    QG_F64 = 1   /* FP64 throughout                                          */
} qg_dtype;

/* Basin geometry and run constants.
 * nx, ny      fine-grid intervals; powers of two, 8 <= nx, ny <= 8192
 *             (FP64: <= 4096 where the grid is solved; larger FP64 elliptic
 *             grids are rejected with QG_ERR_SHAPE).
 * x0..y1      basin extent.  The one-layer experiments of Section 5.1 use
 *             [0,1] x [-1,1]; the two-layer ones of Section 5.2 a square.
 * forcing_amp amplitude a of the double-gyre wind forcing: a sin(pi y)/Ro in
 *             the one-layer vorticity equation (Eq. ge, Section 2.1), and
 *             a sin(2 pi y) on the upper layer of the two-layer model
 *             (Eq. ge-non, Section 2.2).
 * delta       H1/H of the two-layer model (Eq. pv-non); ignored for 1 layer.
 * sigma       bottom-drag coefficient of layer 2 (Eq. ge-non).
 * dt          fixed time step of the TVDRK3 integrator (Section 4.2).
 * flags       reserved, must be 0.                                          */
typedef struct qg_basin {
    int32_t nx, ny;
    double x0, x1, y0, y1;
    double forcing_amp;
    double delta;
    double sigma;
    double dt;
    uint32_t flags;
} qg_basin;

typedef struct qg_ctx* qg_handle;

/* qg_create -- set up a basin (Sections 2 and 3).
 * layers            1 (barotropic vorticity equation, Section 2.1) or 2
 *                   (two-layer QG, Section 2.2).
 * Re, Ro            Reynolds and Rossby numbers.  One layer: the
 *                   dissipation is (1/Re) lap(w) and the beta term
 *                   (1/Ro) J(psi, y) (Eqs. ge, pv, Rhines, Munk).  Two
 *                   layers: A = Ro/Re is the eddy viscosity of Eq. ge-non.
 * Fr                Froude number of Eq. pv-non (two layers; ignored for 1).
 * coarsening_levels 0 <= l <= 4: the elliptic sub-problem is solved on
 *                   level l (Section 3); 0 is the standard full-grid solver.
 *                   The coarse grid must keep at least 8 intervals per
 *                   direction.
 * dtype             QG_F32 or QG_F64.
 * cuda_stream       cudaStream_t on which all work of this handle is
 *                   enqueued (NULL = the legacy default stream).
 * out               receives the handle.  The state starts at rest (w = 0).
 * Errors: QG_ERR_ARG, QG_ERR_SHAPE, QG_ERR_OOM, QG_ERR_CUDA,
 * QG_ERR_NO_DEVICE.  Synchronises the device once (table upload).        */
qg_status qg_create(const qg_basin* basin, int layers, double Re, double Ro,
                    double Fr, int coarsening_levels, qg_dtype dtype,
                    void* cuda_stream, qg_handle* out);

/* qg_destroy -- synchronise the handle's stream and free its device memory.
 * Safe on NULL.                                                            */
qg_status qg_destroy(qg_handle h);

/* qg_set_state / qg_get_state -- copy the prognostic field of `layer`
 * (0-based) into / out of the handle, in the exchange layout of level 0.
 * One layer: the relative vorticity w = (q - y)/Ro (Eq. pv divided by Ro).
 * Two layers: Q_i = q_i - y (Section 4.3).  Walls are implied zero.       */
qg_status qg_set_state(qg_handle h, const void* field, int layer);
qg_status qg_get_state(qg_handle h, void* field, int layer);

/* qg_get_state_async -- as qg_get_state, for a PAGE-LOCKED host buffer,
 * without holding up the handle's later work: the state is repacked on the
 * handle's stream into one of two device staging buffers and copied to the
 * host by DMA on an internal download stream, which the next steps do not
 * wait for (so the copy of step k's result overlaps step k + 1).  The
 * buffer holds the state once qg_synchronize returns (the handle's stream
 * alone does not order it).  Other buffers: the same as qg_get_state.
 * qg_set_state from a page-locked buffer likewise uploads by DMA on an
 * internal stream (the handle's stream waits for it, so its ordering is
 * unchanged), which lets the next input's upload overlap the steps before.
 * Errors: QG_ERR_ARG, QG_ERR_OOM (the staging buffers, on first use).      */
qg_status qg_get_state_async(qg_handle h, void* field, int layer);

/* qg_get_psi -- the fine-grid streamfunction of the current state: the CGP
 * projection of steps (ii)-(iv) of Section 3 (restrict, coarse solve,
 * prolong).  Level-0 exchange layout.                                      */
qg_status qg_get_psi(qg_handle h, void* psi, int layer);

/* qg_set_forcing -- replace the one-layer wind forcing by a fine-grid field
 * F (level-0 exchange layout, added to the vorticity tendency as is).
 * F == NULL restores forcing_amp sin(pi y)/Ro.                            */
qg_status qg_set_forcing(qg_handle h, const void* forcing);

/* qg_poisson_solve -- the elliptic sub-problem on level `level`
 * (0 <= level <= coarsening_levels) with psi = 0 on the walls, by the fast
 * sine-transform solver of Section 4.3: forward DST-I in x and y
 * (Eq. ifft-1), division by the eigenvalues of the 5-point Laplacian
 * (Eq. ialpha), inverse DST-I (Eq. ffft-1).
 * One layer: solves lap_h psi = rhs.
 * Two layers: rhs and psi hold 2 consecutive planes (Q_1, Q_2) and
 * (psi_1, psi_2); solves the coupled system of Eq. sub-pr per mode
 * (Eqs. isub-1/2).                                                         */
qg_status qg_poisson_solve(qg_handle h, const void* rhs, void* psi, int level);

/* qg_restrict -- full-weighting restriction (Eq. res) applied `levels`
 * times, from level 0 to level `levels`.  qg_prolong -- bilinear
 * prolongation (Eq. pro) applied `levels` times, from level `levels` to
 * level 0.  1 <= levels <= coarsening_levels is not required: any level
 * that keeps 2 intervals per direction is accepted.                        */
qg_status qg_restrict(qg_handle h, const void* fine, void* coarse, int levels);
qg_status qg_prolong(qg_handle h, const void* coarse, void* fine, int levels);

/* qg_step -- advance n >= 0 CGPRK3 steps (Section 3.2: TVDRK3 of
 * Section 4.2 whose every stage restricts, solves on the coarse grid,
 * prolongs and updates the fine grid).  Asynchronous; replays a CUDA
 * graph of the step after the first call.                                  */
qg_status qg_step(qg_handle h, int64_t n);

/* qg_diagnostics -- basin-integrated kinetic energy (Section 5.2,
 * E = 1/2 iint |grad psi|^2, one-sided differences on grid edges), the
 * enstrophy Z = 1/2 iint w^2 and max(|psi_x|, |psi_y|) over the interior
 * nodes (the denominator of Eq. dt), for layer 0, accumulated in FP64 in a
 * fixed order (bitwise reproducible).  Any output pointer may be NULL.
 * Host pointers; synchronises the stream.  Returns QG_ERR_NONFINITE when
 * the state holds NaN or Inf.                                              */
qg_status qg_diagnostics(qg_handle h, double* ke, double* enstrophy,
                         double* max_vel);

/* qg_energy_accumulate -- *acc += scale * E, E the basin-integrated kinetic
 * energy of the current state as qg_diagnostics reports it (Section 5.2;
 * psi from the CGP projection, steps (ii)-(iv) of Section 3), added in FP64
 * on the device.  acc: a caller DEVICE pointer to one double.  Asynchronous
 * on the handle's stream (no synchronisation): for sums of the energy over
 * many steps, such as the time-mean energy of an adjoint objective.
 * Errors: QG_ERR_ARG.                                                      */
qg_status qg_energy_accumulate(qg_handle h, double scale, double* acc);

/* Kernel classes of the step, for qg_read_timing.                          */
typedef enum qg_kernel_class {
    QG_K_RESTRICT = 0,   /* restriction (Eq. res), when not fused            */
    QG_K_SOLVE = 1,      /* elliptic solve: sine transforms + eigenvalues    */
    QG_K_PROLONG = 2,    /* prolongation (Eq. pro), when not fused           */
    QG_K_FINE = 3,       /* fine-grid Arakawa / dissipation / forcing / RK   */
    QG_K_CFL = 4,        /* max |grad psi| of the adaptive step (Eq. dt)     */
    QG_K_COUNT = 5
} qg_kernel_class;

/* qg_set_timing -- enable (1) or disable (0) per-kernel timing.  When
 * enabled, the captured step graph records a CUDA event before and after
 * every kernel it launches; this adds event nodes to the graph, so time the
 * whole step with timing disabled.  Re-captures the graph.                 */
qg_status qg_set_timing(qg_handle h, int enable);

/* qg_set_timing_mask -- like qg_set_timing, but only kernels whose class c
 * has bit (1 << c) set in `mask` are bracketed (0 disables timing).  The
 * event nodes between kernels change the step's overlap (a bracketed
 * kernel loses its programmatic early start), so time one class at a time. */
qg_status qg_set_timing_mask(qg_handle h, uint32_t mask);

/* qg_read_timing -- synchronise and return, per kernel class, the summed
 * device time in milliseconds (ms[QG_K_COUNT]) and the number of launches
 * (launches[QG_K_COUNT]) of the most recent step run with timing enabled.  */
qg_status qg_read_timing(qg_handle h, double* ms, int32_t* launches);

/* qg_step_kernel_count -- number of kernels one step launches.             */
qg_status qg_step_kernel_count(qg_handle h, int64_t* count);

/* qg_poisson_solve_noalloc -- the one-layer solve lap_h psi = rhs on an
 * nx x ny-interval grid with spacings dx, dy and psi = 0 on the walls, by
 * the same sine-transform kernels as qg_poisson_solve, for callers that must
 * not allocate device memory (an application that hands out all device
 * memory through its own pool or quota, or a loop where cudaMalloc/cudaFree
 * would synchronise the device).  The paper has no counterpart to this call.
 *
 * It needs no handle and allocates nothing: its workspace lives in one
 * library-owned 32 MiB device array that every GPU loading the library keeps
 * until exit.  The padded grid, its transposed spectrum and the tables must
 * fit in it (for example up to 1024 x 2048 intervals in FP32 or 1024 x 1024
 * in FP64), and one of the shared-memory FFT engines (base radix 4 or 16)
 * must take the grid; other requests return QG_ERR_SHAPE.  rhs and psi are
 * DEVICE pointers in the level-0 exchange layout of that grid; work is
 * enqueued on cuda_stream on the current device, and the call waits for that
 * stream before it returns, so that it can read the solve's error word:
 * a bounded grid-barrier wait that ran out returns QG_ERR_TIMEOUT and leaves
 * psi unwritten.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress): make it before any stream capture starts.
 * All calls share the array: each clears what must start at zero, and calls
 * whose GPU work overlaps (unordered streams) race and give wrong results.  */
qg_status qg_poisson_solve_noalloc(int32_t nx, int32_t ny, double dx, double dy,
                                   qg_dtype dtype, const void* rhs, void* psi,
                                   void* cuda_stream);

/* qg_set_cfl -- adaptive time step (Section 4.2, Eq. dt).  c > 0: every
 * later step uses dt = min(basin.dt, c min(dx, dy) / max|grad psi^n|), the
 * maximum of |psi_x| and |psi_y| (central differences) over the interior
 * fine nodes of the streamfunction of the step's first stage (reduced on the
 * device; the paper states c <= 1); basin.dt caps the step (a flow at rest
 * has no Eq. dt bound).  c = 0: the fixed basin.dt again.  One-layer
 * handles only (QG_ERR_UNSUPPORTED otherwise, or while an adjoint tape is
 * open).  Re-captures the step graph.  Errors: QG_ERR_ARG for c < 0,
 * QG_ERR_CFL for c > 1 (the paper states Eq. dt for c <= 1).              */
qg_status qg_set_cfl(qg_handle h, double c);

/* ---- the elliptic solver of the CGP step (Section 3) -------------------
 * CGP does not depend on the Poisson solver used on the coarse grid; the
 * paper names the V-cycle multigrid as the choice where sine transforms do
 * not apply.                                                               */
typedef enum qg_solver {
    QG_SOLVER_FFT = 0,        /* sine transforms (Section 4.3), the default  */
    QG_SOLVER_MULTIGRID = 1   /* geometric V(2,2) cycles                      */
} qg_solver;

/* qg_set_solver -- the solver of h's steps and of qg_poisson_solve.
 * QG_SOLVER_MULTIGRID: `cycles` (1..64) V(2,2) cycles per solve of
 * lap_h psi = f (red-black Gauss-Seidel smoothing; full weighting, Eq. res,
 * of the residual; bilinear prolongation, Eq. pro, of the correction;
 * grids halved until the shorter side has 2 intervals).  In the step each
 * solve starts from the streamfunction of the previous solve (zero after
 * qg_set_state); qg_poisson_solve starts from zero.  The result is the
 * discrete solution to within the cycles' convergence (about a factor 10
 * per cycle), not to rounding.  One-layer handles whose elliptic grid has
 * sides within a factor 4 of each other and spacings within a factor 2
 * (point smoothing with full coarsening; QG_ERR_UNSUPPORTED otherwise, or
 * while an adjoint tape is open; qg_poisson_solve at a level whose grid
 * does not qualify returns QG_ERR_UNSUPPORTED).  `cycles` is ignored for
 * QG_SOLVER_FFT.  Re-captures the step graph.  Errors: QG_ERR_ARG.        */
qg_status qg_set_solver(qg_handle h, qg_solver kind, int32_t cycles);

/* qg_solve_engine -- which kernel the step's elliptic solves run on (host
 * pointer): chosen when the handle is created by timing whole steps with
 * every candidate that supports the elliptic grid (the QG_SOLVE_ENGINE
 * environment variable forces a supported one; the choice and the stencil
 * tile are cached per grid for the process and, when QG_TUNE_CACHE names a
 * file, in that file).  4 or 16: shared-memory
 * Stockham FFT with base radix 4 or 16; 32, 33, 34: warp-group FFT with 32,
 * 16 or 8 values per thread; 40: the sine sums as dense matrix products on
 * the tensor cores, 3xTF32 (FP32 grids of at most 64 x 128 or 128 x 64
 * intervals with one layer, 64 x 64 with two: both layers' transforms and
 * the coupled solve of Eqs. isub-1/2 per mode); 41: the same products with tcgen05.mma and TMEM
 * accumulators (sides of 16 to 64 intervals); 50: radix-16 FFT passes with the values in
 * registers, one to four sequence pairs per CTA and three launches (one
 * per pass), for elliptic grids of 256 to 8192 intervals a side (4096 in
 * FP64); 0:
 * the multigrid solver (qg_set_solver).  These are
 * implementations of the same sine-transform solve of Section 4.3, equal to
 * rounding.  No device work.  Errors: QG_ERR_ARG.                          */
qg_status qg_solve_engine(qg_handle h, int32_t* engine);

/* qg_stencil_tile -- the tile of the step's fused fine-grid kernel (host
 * pointers): *rows fine rows per CTA (the tile is 64 fine columns wide) and
 * *rows_per_thread (may be NULL) fine rows each thread sweeps.  Chosen when
 * the handle is created by timing whole steps with each tile the build
 * offers for the handle, after the solve engine (qg_solve_engine): one-layer
 * FP32 handles take 128, 64 or 32 rows with 8 rows per thread (16 at
 * l = 4), or 64 or 32 rows with 4 rows per thread at l <= 2 (shorter CTAs:
 * a smaller last wave); FP64 and two-layer handles keep 64 and 128 rows.
 * QG_FINE_ROWS=<rows> or <rows>x<rows per thread> forces an offered tile.
 * Ensemble members keep the default.  The tiles give the same results to
 * rounding.  No device work.  Errors: QG_ERR_ARG.                          */
qg_status qg_stencil_tile(qg_handle h, int32_t* rows, int32_t* rows_per_thread);

/* qg_bounds_check_result -- in a library built with QG_BOUNDS_CHECK (the
 * checked build: every kernel index of the fine stage, the FFT and matrix
 * solves, the transfers, the multigrid solver, the diagnostics and the
 * adjoint is compared with its buffer's extent before the access, and a
 * failed check skips the access instead of trapping):
 * synchronises the device and returns in *site the number of the first
 * check that failed since the last call (0 if none), then clears it.  The
 * paper has no counterpart; this stands in for a memory checker.  Normal
 * builds return QG_ERR_UNSUPPORTED with *site = 0.  Errors: QG_ERR_ARG.   */
qg_status qg_bounds_check_result(int32_t* site);

/* qg_get_time -- model time since creation or the last qg_set_state, and
 * the size of the last step (host pointers; either may be NULL).
 * Synchronises the handle's stream.                                        */
qg_status qg_get_time(qg_handle h, double* t, double* dt_last);

/* ---- time-mean statistics (Section 5.1: the time-mean streamfunction) ---
 * qg_stats_begin -- from now on every step adds psi^n, the streamfunction of
 * its first stage (CGP steps (ii)-(iv) applied to w^n), to an FP64 sum on
 * the device: on the elliptic grid for l >= 1 (prolongation is linear, so
 * the mean of the prolonged fields is the prolonged mean), on the fine grid
 * for l = 0 and for two layers.  Restarts the sum.  Re-captures the step
 * graph.  QG_ERR_UNSUPPORTED while an adjoint tape is open.               */
qg_status qg_stats_begin(qg_handle h);

/* qg_stats_mean_psi -- the mean of psi^n over the steps since
 * qg_stats_begin, prolonged to the fine grid, into the caller's device
 * buffer (exchange layout, handle dtype; NULL to read only the count) for
 * `layer`; *count (may be NULL) = number of steps averaged.
 * Errors: QG_ERR_ARG when no step has been accumulated.                    */
qg_status qg_stats_mean_psi(qg_handle h, void* psi_mean, int layer, int64_t* count);

/* qg_stats_mean_q -- the time-mean potential vorticity over the same steps
 * as qg_stats_mean_psi (the sums of the states w^n or Q_i^n are kept beside
 * those of psi^n): one layer q = Ro w + y (Eq. pv with (delta_I/L)^2 = Ro,
 * Eq. Rhines), two layers q_i = Q_i + y (Section 4.3); fine grid, exchange
 * layout, handle dtype, into the caller's device buffer (NULL to read only
 * the count).  Errors: QG_ERR_ARG when no step has been accumulated.     */
qg_status qg_stats_mean_q(qg_handle h, void* q_mean, int layer, int64_t* count);

/* qg_stats_end -- stop accumulating (the sum is kept).                     */
qg_status qg_stats_end(qg_handle h);

/* qg_inject_fault -- failure-detection test switch (the paper has no
 * counterpart).  kind = QG_FAULT_BARRIER_STALL makes every later elliptic
 * solve of the handle wait at its first grid barrier for one arrival more
 * than the grid has, so the wait runs out of its bound (about a second),
 * the kernel sets the handle's error flag and returns; the next
 * qg_synchronize or qg_diagnostics returns QG_ERR_TIMEOUT and clears the
 * flag.  Results computed meanwhile are garbage.  QG_FAULT_NONE restores
 * normal operation.  No memory outside the handle's buffers is touched and
 * the CUDA context stays usable.  Re-captures the step graph.  Ensemble
 * members solve with three plain launches and no grid barrier: there the
 * switch has no effect.
 * Errors: QG_ERR_ARG for a NULL handle or an unknown kind.                 */
typedef enum qg_fault {
    QG_FAULT_NONE = 0,
    QG_FAULT_BARRIER_STALL = 1
} qg_fault;
qg_status qg_inject_fault(qg_handle h, int kind);

/* ---- discrete adjoint (one layer) ------------------------------------------
 * The paper has no adjoint.  These calls give the exact transpose of the
 * Jacobian of the discrete CGPRK3 step of Section 3.2 (restriction Eq. res,
 * Poisson solve Section 4.3, prolongation Eq. pro, Arakawa Jacobian
 * Eq. ja1, TVDRK3 Eq. TVDRK), for gradients of functionals of the
 * trajectory, such as a time-mean kinetic energy (Section 5.2), with
 * respect to the state and to the wind-forcing field F.  With psi = A w,
 * A = P^l S R^l (symmetric), the transposed right-hand side is
 *   G_w^T lam = J(psi, lam) + (1/Re) lap lam - A[J(w, lam) - (1/Ro) J(lam, y)],
 * using that J(p, .) and J(., y) are skew-symmetric with zero walls.
 *
 * Usage: qg_tape_begin records the current state as tape time 0; every
 * later qg_step(h, n) appends n steps (at most max_steps in all).  The
 * reverse cursor starts at the last recorded time t; qg_adjoint_step moves
 * it back, qg_energy_gradient reads the state at it.  The forward states
 * are stored every `every` steps (every = 1 keeps all of them; a 256 x 512
 * FP32 state is 0.6 MB, a 2048 x 4096 one 34 MB) and the others are
 * recomputed per segment with the handle's own step graph.  While a tape
 * is being reversed with every > 1 the handle's state serves as scratch;
 * qg_tape_end puts back the state the handle had when the reversal began.
 * One-layer handles only (QG_ERR_UNSUPPORTED for two layers).            */

/* qg_tape_begin -- start recording.  every >= 1, max_steps >= 1.
 * Errors: QG_ERR_ARG, QG_ERR_OOM, QG_ERR_UNSUPPORTED.                      */
qg_status qg_tape_begin(qg_handle h, int64_t every, int64_t max_steps);

/* qg_tape_end -- stop recording, free the tape, restore the state (see
 * above).  Safe without a tape.                                            */
qg_status qg_tape_end(qg_handle h);

/* qg_adjoint_step -- reverse n steps from the cursor t (n <= t): on entry
 * lambda holds dJ/dw at time t, on return dJ/dw at time t - n through those
 * steps; dJdF += dJ/dF through them.  lambda and dJdF are caller device
 * buffers in the exchange layout and the handle's dtype.  Objective terms at
 * intermediate times are added between calls (qg_energy_gradient).
 * Errors: QG_ERR_ARG (no tape, n out of range, NULL buffers).              */
qg_status qg_adjoint_step(qg_handle h, int64_t n, void* lambda, void* dJdF);

/* qg_energy_gradient -- g += scale * dE/dw at the state of tape time t (the
 * cursor), E the kinetic energy of psi = A w (as qg_diagnostics reports it):
 * dE/dw = A(-dx dy lap psi).  g: caller device buffer, exchange layout.    */
qg_status qg_energy_gradient(qg_handle h, double scale, void* g);

/* ---- ensembles of basins --------------------------------------------------
 * Many independent one-layer basins (Section 2.1), each with its own grid,
 * Re, Ro, forcing amplitude, dt and CGP level (Section 3), stepped together:
 * one CUDA graph per ensemble step.  Members whose elliptic grids have the
 * same shape and spacing form a group; per TVDRK3 stage a group runs one
 * batched solve for all its members and one batched fused fine stage per
 * fine level (members' tiles side by side in one launch), and each group's
 * chain is a branch of its own in the graph.  A group's solve engine is
 * picked when the ensemble is created, by timing whole group steps with
 * each engine that batches its grid (the members' buffers are zeroed
 * afterwards); the choice is cached for the process and, when the
 * QG_TUNE_CACHE environment variable names a file, in that file.  With the
 * same solve engine and tile the results are bitwise those of stand-alone
 * handles.  A group with a member on the multigrid solver runs its
 * members' own solves.  The
 * paper runs one basin at a time; the ensemble is this library's way of
 * filling a GPU with small basins.                                         */
typedef struct qg_ensemble_s* qg_ensemble;

/* qg_ensemble_create -- `count` (1..4096) members; basins[i], Re[i], Ro[i],
 * levels[i] as for qg_create with layers = 1 and Fr = 0.  All members share
 * `dtype` and `cuda_stream`.  Builds the step graph (group engines timed on
 * the device, see above); member states start at zero.
 * Errors: as qg_create for the first failing member (nothing is kept),
 * QG_ERR_CUDA if the graph cannot be built, QG_ERR_ARG for NULL arrays or
 * a bad count.                                                             */
qg_status qg_ensemble_create(const qg_basin* basins, const double* Re, const double* Ro,
                             const int* levels, int count, qg_dtype dtype,
                             void* cuda_stream, qg_ensemble* out);

/* qg_ensemble_member -- the handle of member `index`, for qg_set_state,
 * qg_get_state, qg_get_psi, qg_set_forcing, qg_diagnostics and
 * qg_synchronize.  The ensemble owns it: do not qg_destroy it.  qg_step on a
 * member steps that member alone.                                          */
qg_status qg_ensemble_member(qg_ensemble e, int index, qg_handle* out);

/* qg_ensemble_step -- n steps of every member, asynchronous on the
 * ensemble's stream (one graph launch per step).                           */
qg_status qg_ensemble_step(qg_ensemble e, int64_t n);

/* qg_ensemble_kernel_count -- kernels one ensemble step launches (rebuilds
 * the graph first if a member's own step changed).                         */
qg_status qg_ensemble_kernel_count(qg_ensemble e, int64_t* count);

/* qg_ensemble_synchronize -- wait for the ensemble's work; returns the
 * first error of any member (bounded-wait timeouts included).              */
qg_status qg_ensemble_synchronize(qg_ensemble e);

/* qg_ensemble_destroy -- frees the members and the graph; safe on NULL.    */
qg_status qg_ensemble_destroy(qg_ensemble e);

/* qg_synchronize -- wait for the handle's work; returns any latched error. */
qg_status qg_synchronize(qg_handle h);

/* qg_status_string -- static text for a status code.                       */
const char* qg_status_string(qg_status s);

/* qg_last_error -- the latched error of the handle (QG_OK if none); reading
 * it clears it.                                                            */
qg_status qg_last_error(qg_handle h);

#ifdef __cplusplus
}
#endif

#endif /* QG_H */
