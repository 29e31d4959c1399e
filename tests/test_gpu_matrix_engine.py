"""GPU parity of the matrix-form elliptic solve (engine 40): the sine sums
of Section 4.3 (Eqs. ffft-1/2, ifft-1/2) as dense products with the sine
matrices on the tensor cores, 3xTF32 with FP32 accumulation, and the
eigenvalue division of Eq. ialpha between them.  Same tolerances as the FFT
engines: relative L2 <= 2e-6 for a solve in FP32, <= 1e-4 after 100 FP32
steps."""
import numpy as np
import pytest

from oracle import qg_oracle as O
from paper_1308_3290_gb300 import inputs, qg
from tests.gpu_util import rel_l2, require_gpu, to_np

pytestmark = pytest.mark.gpu

MATRIX = 40


def forced_basin(monkeypatch, nx, ny, levels, **kw):
    monkeypatch.setenv("QG_SOLVE_ENGINE", str(MATRIX))
    b = qg.Basin(nx, ny, Re=kw.pop("Re", 200.0), Ro=kw.pop("Ro", 0.0016), levels=levels,
                 dt=kw.pop("dt", 1e-4), dtype="f32", **kw)
    assert qg.qg_solve_engine(b.h) == MATRIX
    return b


@pytest.mark.parametrize("nx,ny,y0,y1", [
    (8, 8, -1.0, 1.0), (8, 16, -1.0, 1.0), (16, 8, -0.5, 0.5), (16, 32, -1.0, 1.0),
    (32, 32, -0.5, 0.5), (32, 64, -1.0, 1.0), (64, 64, -0.5, 0.5), (64, 128, -1.0, 1.0),
    (128, 64, -0.5, 0.5), (16, 128, -1.0, 1.0), (128, 16, -1.0, 1.0),
])
def test_matrix_solve_parity(nx, ny, y0, y1, monkeypatch):
    require_gpu()
    b = forced_basin(monkeypatch, nx, ny, 0, y0=y0, y1=y1)
    for rhs in (inputs.smooth_field(nx, ny, seed=nx + ny, noise=0.3),
                inputs.random_field(nx, ny, seed=nx * ny)):
        got = to_np(b.poisson_solve(rhs))
        ref = O.poisson_solve(rhs, nx, ny, 1.0 / nx, (y1 - y0) / ny)
        assert rel_l2(got, ref) <= 2e-6, (nx, ny, rel_l2(got, ref))
        # the wall nodes of psi stay zero
        assert np.isfinite(got).all()
    b.close()


def lap_h(psi, dx, dy):
    """The 5-point Laplacian whose eigenvalues Eq. ialpha gives, psi = 0 on
    the walls, in FP64."""
    p = np.pad(psi.astype(np.float64), 1)
    return ((p[1:-1, 2:] - 2 * p[1:-1, 1:-1] + p[1:-1, :-2]) / dx ** 2
            + (p[2:, 1:-1] - 2 * p[1:-1, 1:-1] + p[:-2, 1:-1]) / dy ** 2)


def test_matrix_solve_of_discrete_eigenmodes(monkeypatch):
    """A discrete eigenmode rhs = lambda_kl sin sin comes back as the mode
    (Eq. ialpha).  Low and middle modes: forward error at FP32 rounding.
    The highest mode: its solution is ill-conditioned in FP32 (the rounding
    of the rhs itself, amplified by lambda_max / lambda_min, gives a forward
    error of a few 1e-6), so its backward error, the residual against the
    FP32 rhs, is the check."""
    require_gpu()
    nx, ny = 64, 128
    dx, dy = 1.0 / nx, 2.0 / ny
    b = forced_basin(monkeypatch, nx, ny, 0)
    I = np.arange(1, nx)[None, :]
    J = np.arange(1, ny)[:, None]
    for k, l in ((1, 1), (1, 2), (17, 40), (nx - 1, ny - 1)):
        mode = np.sin(np.pi * k * I / nx) * np.sin(np.pi * l * J / ny)
        lam = (2 * np.cos(np.pi * k / nx) - 2) / dx**2 + (2 * np.cos(np.pi * l / ny) - 2) / dy**2
        rhs = (lam * mode).astype(np.float32)
        got = to_np(b.poisson_solve(rhs))
        if k < nx - 1:
            assert rel_l2(got, mode) <= 2e-6, (k, l, rel_l2(got, mode))
        else:
            res = rel_l2(lap_h(got, dx, dy), rhs.astype(np.float64))
            assert res <= 1e-5, (k, l, res)
    b.close()


@pytest.mark.parametrize("nx,ny,levels", [(64, 128, 0), (64, 128, 1), (128, 256, 2),
                                          (128, 128, 1)])
def test_matrix_engine_in_the_step(nx, ny, levels, monkeypatch):
    """100 FP32 CGP steps (the restriction's partial planes feed the matrix
    solve at l >= 1) against the oracle's FP64 steps."""
    require_gpu()
    w0 = inputs.perturbation(nx, ny, seed=11) * 50.0
    ob = O.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=levels, dt=5e-5)
    ref = O.run(w0, ob, 100)
    b = forced_basin(monkeypatch, nx, ny, levels, dt=5e-5)
    b.set_state(w0)
    b.step(100)
    got = to_np(b.state())
    assert rel_l2(got, ref) <= 1e-4, rel_l2(got, ref)
    b.close()


def test_matrix_engine_unsupported_grids_fall_back(monkeypatch):
    """Grids past the engine's shared memory (one layer beyond 64 x 128, two
    layers beyond 64 x 64) and FP64 handles keep an FFT engine although the
    matrix engine is requested."""
    require_gpu()
    monkeypatch.setenv("QG_SOLVE_ENGINE", str(MATRIX))
    cases = [dict(nx=128, ny=128, dtype="f32"), dict(nx=64, ny=128, dtype="f64"),
             dict(nx=128, ny=128, dtype="f32", layers=2, Fr=0.087, delta=0.2, sigma=1.43e-3,
                  y0=-0.5, y1=0.5)]
    for c in cases:
        b = qg.Basin(Re=200.0, Ro=0.0016, levels=0, dt=1e-4, **c)
        assert qg.qg_solve_engine(b.h) in (4, 16, 32, 33, 34)
        b.close()


def test_matrix_engine_in_an_ensemble_equals_standalone_handles(monkeypatch):
    """Ensemble members on the matrix engine: bitwise the stand-alone
    handles' steps; the ensemble solves each group of equal elliptic grids
    (here 32 x 64 for three members at levels 0, 1, 2, and 32 x 16 for one)
    in one launch with one CTA per member, and sweeps each level's members
    of a group in one launch."""
    require_gpu()
    monkeypatch.setenv("QG_SOLVE_ENGINE", str(MATRIX))
    monkeypatch.setenv("QG_FINE_ROWS", "64")   # the members' (batched) tile
    members = [
        dict(nx=32, ny=64, Re=200.0, Ro=0.0016, levels=0, dt=1e-4, amp=1.0),
        dict(nx=64, ny=128, Re=312.5, Ro=0.0025, levels=1, dt=1e-4, amp=1.3),
        dict(nx=128, ny=256, Re=800.0, Ro=0.0016, levels=2, dt=5e-5, amp=0.5),
        dict(nx=256, ny=128, Re=200.0, Ro=0.0016, levels=3, dt=2e-5, amp=1.0),
    ]
    ens = qg.Ensemble(members, dtype="f32")
    solo = [qg.Basin(m["nx"], m["ny"], Re=m["Re"], Ro=m["Ro"], levels=m["levels"], dt=m["dt"],
                     amp=m["amp"], dtype="f32") for m in members]
    w = [inputs.perturbation(m["nx"], m["ny"], seed=70 + i) * 40.0 for i, m in enumerate(members)]
    for i in range(len(members)):
        assert qg.qg_solve_engine(ens.member(i).h) == MATRIX
        assert qg.qg_solve_engine(solo[i].h) == MATRIX
        ens.member(i).set_state(w[i])
        solo[i].set_state(w[i])
    ens.step(10)
    for b in solo:
        b.step(10)
    ens.synchronize()
    for i, b in enumerate(solo):
        b.synchronize()
        assert np.array_equal(to_np(ens.member(i).state()), to_np(b.state())), i
    assert sum(qg.qg_step_kernel_count(b.h) for b in solo) == 3 * 2 * len(members)
    assert ens.kernel_count() == 3 * (2 + 4)
    m = members[1]
    ref = O.run(w[1], O.Basin(m["nx"], m["ny"], Re=m["Re"], Ro=m["Ro"], levels=m["levels"],
                              dt=m["dt"], amp=m["amp"]), 10)
    assert rel_l2(to_np(ens.member(1).state()), ref) <= 1e-4
    for b in solo:
        b.close()
    ens.close()


@pytest.mark.parametrize("nx,ny", [(16, 16), (32, 32), (64, 64), (32, 64)])
def test_two_layer_matrix_solve_parity(nx, ny, monkeypatch):
    """Both layers' transforms and the coupled solve of Eqs. isub-1/2 per
    mode in the matrix form, against the oracle's two-layer elliptic solve
    (square basin of Section 2.2 and an N x 2N one)."""
    require_gpu()
    p = dict(Ro=2.49e-4, Fr=0.087, delta=0.2, sigma=1.43e-3)
    b = forced_basin(monkeypatch, nx, ny, 0, Re=697.16, dt=1e-5, layers=2, y0=-0.5, y1=0.5, **p)
    Q1 = inputs.smooth_field(nx, ny, seed=1, noise=0.1)
    Q2 = inputs.smooth_field(nx, ny, seed=2, noise=0.1)
    got = to_np(b.poisson_solve(np.stack([Q1, Q2])))
    r1, r2 = O.elliptic_two_layer(Q1, Q2, nx, ny, 1 / nx, 1 / ny, p["Ro"], p["Fr"], p["delta"])
    assert rel_l2(got[0], r1) <= 1e-5, rel_l2(got[0], r1)
    assert rel_l2(got[1], r2) <= 1e-5, rel_l2(got[1], r2)
    b.close()


@pytest.mark.parametrize("levels", [0, 1])
def test_two_layer_matrix_engine_in_the_step(levels, monkeypatch):
    """20 FP32 steps of the two-layer basin (Table 2 Experiment 1 parameters,
    64 x 64) on the matrix engine against the oracle's FP64 steps."""
    require_gpu()
    p = dict(Ro=2.49e-4, Fr=0.087, delta=0.2, sigma=1.43e-3)
    A = 3.57e-7
    Q1 = inputs.smooth_field(64, 64, seed=1, amp=0.05, noise=0.01)
    Q2 = inputs.smooth_field(64, 64, seed=2, amp=0.02, noise=0.01)
    ob = O.TwoLayer(64, 64, A=A, levels=levels, dt=1e-4, **p)
    a1, a2 = O.embed(Q1), O.embed(Q2)
    for _ in range(20):
        a1, a2 = O.cgprk3_step_two_layer(a1, a2, ob)
    b = forced_basin(monkeypatch, 64, 64, levels, Re=p["Ro"] / A, dt=1e-4, layers=2, y0=-0.5,
                     y1=0.5, **p)
    b.set_state(Q1, 0)
    b.set_state(Q2, 1)
    b.step(20)
    assert rel_l2(to_np(b.state(0)), O.interior(a1)) <= 1e-4
    assert rel_l2(to_np(b.state(1)), O.interior(a2)) <= 1e-4
    b.close()
