// The matrix-form elliptic solve (solve_mtx.cu): declarations for the host
// code that builds its tables and picks it as a solve engine.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "qg_internal.cuh"

namespace qg {

// Engine number of the matrix-form solve among the autotuner's candidates
// (the FFT engines are 4, 16 and 32-34).
constexpr int kMatrixEngine = 40;

// FP32 elliptic grids (one layer, or two: both layers' transforms and the
// coupled solve of Eqs. isub-1/2) whose sine matrices and work arrays fit
// in 200 KB of one CTA's shared memory (Mx, My powers of two): one layer up
// to 64 x 128 or 128 x 64 intervals (156 KB), two layers up to 64 x 64.
bool mtx_supports(int mx, int my, size_t esz, int layers);
size_t mtx_smem_bytes(int mx, int my, int layers);

// The constant table of one elliptic grid: S_x (padded), S_y (padded) and
// the scaled inverse eigenvalues (2/Mx)(2/My)/lambda_kl of Eq. ialpha, in
// the layout the kernel copies into shared memory; FP64-evaluated, stored
// FP32.  mtx_table_floats(mx, my) entries.
size_t mtx_table_floats(int mx, int my);
void mtx_table(int mx, int my, double dx, double dy, float* out);

// The solve of one level: P as for launch_solve (one layer, FP32; P.split
// is ignored: one single-CTA launch either way), tab the device copy of
// mtx_table.
cudaError_t launch_solve_mtx(const SolveParams<float>& P, const float* tab, cudaStream_t s);

// The same solve with tcgen05.mma and TMEM accumulators (solve_tc.cu):
// one-layer FP32 grids with sides of 16, 32 or 64 intervals; one CTA per
// grid (per member for a batch).  Its table holds the split sine matrices
// in the kernel's shared-memory layout, then the scaled inverse
// eigenvalues; tc_table_floats(mx, my) entries, FP64-evaluated.
constexpr int kTcEngine = 41;
bool tc_supports(int mx, int my, size_t esz, int layers);
size_t tc_table_floats(int mx, int my);
void tc_table(int mx, int my, double dx, double dy, float* out);
cudaError_t launch_solve_tc(const SolveParams<float>& P, const float* tab, cudaStream_t s);
int bounds_site_tc();

}  // namespace qg
