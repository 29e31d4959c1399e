"""GPU parity of the elliptic solver (qg_poisson_solve, Section 4.3) with
the oracle: relative L2 <= 1e-12 in FP64 and <= 2e-6 in FP32, on seeded
inputs, from the smallest grid to the 2048 x 4096 full-grid solve."""
import numpy as np
import pytest

from oracle import qg_oracle as O
from paper_1308_3290_gb300 import inputs, qg
from tests.gpu_util import rel_l2, require_gpu, to_np

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6}


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny,y0,y1", [
    (8, 8, -1.0, 1.0), (8, 16, -1.0, 1.0), (16, 8, -0.5, 0.5), (64, 128, -1.0, 1.0),
    (128, 64, -0.5, 0.5), (32, 2048, -1.0, 1.0), (2048, 16, -1.0, 1.0),
    (512, 1024, -1.0, 1.0),
])
def test_poisson_parity(dtype, nx, ny, y0, y1):
    require_gpu()
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=0, dt=1e-4, dtype=dtype, y0=y0, y1=y1)
    rhs = inputs.smooth_field(nx, ny, seed=nx + ny, noise=0.3)
    got = to_np(b.poisson_solve(rhs, level=0))
    ref = O.poisson_solve(rhs, nx, ny, 1.0 / nx, (y1 - y0) / ny)
    assert rel_l2(got, ref) <= TOL[dtype]
    b.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_poisson_parity_white_noise(dtype):
    require_gpu()
    nx, ny = 256, 512
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=0, dt=1e-4, dtype=dtype)
    rhs = inputs.random_field(nx, ny, seed=5)
    got = to_np(b.poisson_solve(rhs))
    ref = O.poisson_solve(rhs, nx, ny, 1.0 / nx, 2.0 / ny)
    assert rel_l2(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("level", [1, 2])
def test_poisson_on_coarse_levels(level):
    require_gpu()
    nx, ny = 128, 256
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=2, dt=1e-4, dtype="f64")
    mx, my = nx >> level, ny >> level
    rhs = inputs.smooth_field(mx, my, seed=level, noise=0.1)
    got = to_np(b.poisson_solve(rhs, level=level))
    ref = O.poisson_solve(rhs, mx, my, 1.0 / mx, 2.0 / my)
    assert rel_l2(got, ref) <= 1e-12


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_full_size_solves(dtype):
    """The elliptic grid of the 2048 x 4096, l = 2 workload (512 x 1024) and
    the full-grid (l = 0) 2048 x 4096 solve."""
    require_gpu()
    for lv in (2, 0):
        nx, ny = 2048 >> lv, 4096 >> lv
        b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=0, dt=1e-4, dtype=dtype)
        rhs = inputs.smooth_field(nx, ny, seed=7, noise=0.2)
        got = to_np(b.poisson_solve(rhs))
        ref = O.poisson_solve(rhs, nx, ny, 1.0 / nx, 2.0 / ny)
        assert rel_l2(got, ref) <= TOL[dtype], (lv, rel_l2(got, ref))
        b.close()


def test_two_layer_solve_parity():
    require_gpu()
    nx, ny = 64, 64
    for dtype in ("f64", "f32"):
        b = qg.Basin(nx, ny, Re=697.16, Ro=2.49e-4, Fr=0.087, delta=0.2, sigma=1.43e-3,
                     levels=0, dt=1e-5, dtype=dtype, layers=2, y0=-0.5, y1=0.5)
        Q1 = inputs.smooth_field(nx, ny, seed=1, noise=0.1)
        Q2 = inputs.smooth_field(nx, ny, seed=2, noise=0.1)
        got = to_np(b.poisson_solve(np.stack([Q1, Q2])))
        r1, r2 = O.elliptic_two_layer(Q1, Q2, nx, ny, 1 / nx, 1 / ny, 2.49e-4, 0.087, 0.2)
        assert rel_l2(got[0], r1) <= TOL[dtype] * 5
        assert rel_l2(got[1], r2) <= TOL[dtype] * 5
        b.close()


@pytest.mark.parametrize("engine", ["4", "16", "32", "33", "34"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_both_fft_engines(engine, dtype, monkeypatch):
    """The solve has five FFT schedules (shared-memory engine with base
    radix 4 or 16, warp-group engine with 32, 16 or 8 values per thread)
    chosen by the autotuner; each must meet the same tolerance (the matrix
    form of small grids has its own tests)."""
    require_gpu()
    monkeypatch.setenv("QG_SOLVE_ENGINE", engine)
    shapes = [(64, 128), (512, 1024), (2048, 256)]
    if engine in ("32", "33", "34"):
        shapes += [(16, 16), (32, 64), (256, 32), (4096, 64), (1024, 2048)]
    for nx, ny in shapes:
        b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=0, dt=1e-4, dtype=dtype)
        rhs = inputs.smooth_field(nx, ny, seed=nx, noise=0.3)
        got = to_np(b.poisson_solve(rhs))
        ref = O.poisson_solve(rhs, nx, ny, 1.0 / nx, 2.0 / ny)
        assert rel_l2(got, ref) <= TOL[dtype], (nx, ny, rel_l2(got, ref))
        b.close()


@pytest.mark.parametrize("engine", ["32", "33", "34"])
@pytest.mark.parametrize("levels", [0, 1, 2])
def test_warp_engine_in_the_step(levels, engine, monkeypatch):
    """100 FP64 steps with a warp-group engine forced, one layer and two."""
    require_gpu()
    monkeypatch.setenv("QG_SOLVE_ENGINE", engine)
    nx, ny = 64, 128
    w0 = inputs.perturbation(nx, ny, seed=3) * 50.0
    ob = O.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=levels, dt=1e-4)
    ref = O.run(w0, ob, 100)
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=levels, dt=1e-4, dtype="f64")
    b.set_state(w0)
    b.step(100)
    assert rel_l2(to_np(b.state()), ref) <= 1e-12
    b.close()
    if levels <= 1:
        p = dict(Ro=2.49e-4, Fr=0.087, delta=0.2, sigma=1.43e-3)
        A = 3.57e-7
        Q1 = inputs.smooth_field(64, 64, seed=1, amp=0.05, noise=0.01)
        Q2 = inputs.smooth_field(64, 64, seed=2, amp=0.02, noise=0.01)
        ob2 = O.TwoLayer(64, 64, A=A, levels=levels, dt=1e-4, **p)
        a1, a2 = O.embed(Q1), O.embed(Q2)
        for _ in range(20):
            a1, a2 = O.cgprk3_step_two_layer(a1, a2, ob2)
        b2 = qg.Basin(64, 64, Re=p["Ro"] / A, levels=levels, dt=1e-4, dtype="f64", layers=2,
                      y0=-0.5, y1=0.5, **p)
        b2.set_state(Q1, 0)
        b2.set_state(Q2, 1)
        b2.step(20)
        assert rel_l2(to_np(b2.state(0)), O.interior(a1)) <= 1e-11
        assert rel_l2(to_np(b2.state(1)), O.interior(a2)) <= 1e-11
        b2.close()
