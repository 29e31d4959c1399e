"""Edge cases of the CUDA path: the largest grids the ABI accepts (checked
through the exact discrete eigenmodes of the 5-point Laplacian, which the
solve must return to rounding at any size), the smallest basin and the
deepest coarsening, and the degenerate flow (rest, no forcing)."""
import numpy as np
import pytest

from oracle import qg_oracle as O
from paper_1308_3290_gb300 import inputs, qg
from tests.gpu_util import rel_l2, require_gpu, to_np

pytestmark = pytest.mark.gpu


def mode(nx, ny, k, l):
    """sin(pi k i/nx) sin(pi l j/ny) on the interior nodes."""
    i = np.arange(1, nx)
    j = np.arange(1, ny)
    return np.sin(np.pi * l * j / ny)[:, None] * np.sin(np.pi * k * i / nx)[None, :]


def eigenvalue(nx, ny, dx, dy, k, l):
    return ((2 * np.cos(np.pi * k / nx) - 2) / dx ** 2
            + (2 * np.cos(np.pi * l / ny) - 2) / dy ** 2)


def lap_h(psi, dx, dy):
    """The 5-point Laplacian (the operator whose eigenvalues Eq. ialpha gives) with psi = 0 on the
    boundary, in FP64."""
    p = np.pad(psi.astype(np.float64), 1)
    return ((p[1:-1, 2:] - 2 * p[1:-1, 1:-1] + p[1:-1, :-2]) / dx ** 2
            + (p[2:, 1:-1] - 2 * p[1:-1, 1:-1] + p[:-2, 1:-1]) / dy ** 2)


@pytest.mark.parametrize("nx,ny,dtype,fwd,bwd", [
    (8192, 8192, "f32", 2e-6, 1e-5), (8192, 64, "f32", 2e-6, 1e-5),
    (16, 8192, "f32", 2e-6, 1e-5),
    (4096, 4096, "f64", 1e-12, 1e-13), (4096, 16, "f64", 1e-12, 1e-13)])
def test_largest_grids_return_exact_eigenmodes(nx, ny, dtype, fwd, bwd):
    """lap_h of a discrete sine mode is lambda_kl times the mode, so the
    solve of lambda_kl * mode must return the mode.  The largest grids: 8192
    intervals per direction in FP32, 4096 in FP64 (larger FP64 grids are
    rejected with QG_ERR_SHAPE: no FFT engine's shared memory holds them).

    The lowest mode is checked by its forward error.  For a mode far up the
    spectrum the forward error is the rounding of the right-hand side (and of
    the transforms) amplified by lambda_kl / lambda_11, up to 10^7 here, so
    those modes are checked by the backward error instead: the residual
    lap_h(psi) - rhs relative to rhs, which a stable solve keeps at a few
    units of rounding at any size.  (For the lowest mode the residual is the
    wrong measure the other way round: lap_h amplifies the last-bit rounding
    of psi by |lambda_max| / |lambda_11|.)"""
    require_gpu()
    dx, dy = 1.0 / nx, 2.0 / ny
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=0, dt=1e-6, dtype=dtype)
    for n, (k, l) in enumerate(((1, 2), (nx // 3, ny // 5), (nx - 3, ny - 5))):
        want = mode(nx, ny, k, l)
        rhs = eigenvalue(nx, ny, dx, dy, k, l) * want
        got = to_np(b.poisson_solve(rhs))
        if n == 0:
            assert rel_l2(got, want) <= fwd, (k, l, rel_l2(got, want))
        else:
            rhs_t = rhs.astype(np.float32 if dtype == "f32" else np.float64)
            res = rel_l2(lap_h(got, dx, dy), rhs_t.astype(np.float64))
            assert res <= bwd, (k, l, res)
    b.close()


def test_smallest_basin_and_deepest_coarsening():
    """8 x 8 intervals (the smallest grid), and 128 x 128 with l = 4 (elliptic
    grid 8 x 8), each 20 FP64 steps against the oracle."""
    require_gpu()
    for nx, ny, lv in ((8, 8, 0), (128, 128, 4), (256, 128, 4)):
        w0 = inputs.perturbation(nx, ny, seed=nx + lv) * 50.0
        ob = O.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=lv, dt=1e-4)
        ref = O.run(w0, ob, 20)
        b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=lv, dt=1e-4, dtype="f64")
        b.set_state(w0)
        b.step(20)
        assert rel_l2(to_np(b.state()), ref) <= 1e-12, (nx, ny, lv)
        b.close()


def test_rest_without_forcing_stays_at_rest():
    """With zero forcing a basin at rest stays exactly at rest (every term of
    G vanishes), in both precisions and at the benchmark's level."""
    torch = require_gpu()
    for dtype in ("f32", "f64"):
        b = qg.Basin(256, 512, Re=200.0, Ro=0.0016, levels=2, dt=1e-4, dtype=dtype, amp=0.0)
        b.set_state(np.zeros((511, 255)))
        b.step(10)
        assert float(torch.count_nonzero(b.state())) == 0.0
        ke, z, u = b.diagnostics()
        assert ke == 0.0 and z == 0.0 and u == 0.0
        b.close()


def test_rejected_requests_leave_no_handle():
    """Shapes the library does not take come back as errors, not faults."""
    require_gpu()
    for nx, ny, lv in ((16384, 64, 0), (64, 48, 0), (64, 128, 4)):
        with pytest.raises(qg.QGError):
            qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=lv, dt=1e-4)


def test_fp64_beyond_4096_is_rejected():
    require_gpu()
    with pytest.raises(qg.QGError):
        qg.Basin(8192, 64, Re=200.0, Ro=0.0016, levels=0, dt=1e-4, dtype="f64")
