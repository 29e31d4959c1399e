"""GPU parity of engine 41: the matrix-form elliptic solve of Section 4.3
(the sine sums of Eqs. ffft-1/2, ifft-1/2 as products with the sine
matrices, the division of Eq. ialpha between them) on the tensor cores with
tcgen05.mma, TMEM accumulators and 3xTF32 operands.  The tolerances of the
other engines: relative L2 <= 2e-6 for an FP32 solve, <= 1e-4 after 100
FP32 steps; an ensemble is bitwise its stand-alone handles."""
import numpy as np
import pytest

from oracle import qg_oracle as O
from paper_1308_3290_gb300 import inputs, qg
from tests.gpu_util import rel_l2, require_gpu, to_np

pytestmark = pytest.mark.gpu

TC = 41


def forced_basin(monkeypatch, nx, ny, levels, engine=TC, **kw):
    monkeypatch.setenv("QG_SOLVE_ENGINE", str(engine))
    b = qg.Basin(nx, ny, Re=kw.pop("Re", 200.0), Ro=kw.pop("Ro", 0.0016), levels=levels,
                 dt=kw.pop("dt", 1e-4), dtype="f32", **kw)
    assert qg.qg_solve_engine(b.h) == engine
    return b


@pytest.mark.parametrize("nx,ny,y0,y1", [
    (16, 16, -1.0, 1.0), (16, 32, -1.0, 1.0), (32, 16, -0.5, 0.5), (32, 32, -0.5, 0.5),
    (32, 64, -1.0, 1.0), (64, 32, -1.0, 1.0), (64, 64, -0.5, 0.5), (16, 64, -1.0, 1.0),
])
def test_tc_solve_parity(nx, ny, y0, y1, monkeypatch):
    require_gpu()
    b = forced_basin(monkeypatch, nx, ny, 0, y0=y0, y1=y1)
    for rhs in (inputs.smooth_field(nx, ny, seed=nx + ny, noise=0.3),
                inputs.random_field(nx, ny, seed=nx * ny)):
        got = to_np(b.poisson_solve(rhs))
        ref = O.poisson_solve(rhs, nx, ny, 1.0 / nx, (y1 - y0) / ny)
        assert rel_l2(got, ref) <= 2e-6, (nx, ny, rel_l2(got, ref))
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    b.close()


def test_tc_solve_of_discrete_eigenmodes(monkeypatch):
    """Discrete eigenmodes come back as themselves (Eq. ialpha): forward
    error for the low and middle modes, the residual for the highest."""
    require_gpu()
    nx, ny = 64, 64
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
            p = np.pad(got, 1)
            lap = ((p[1:-1, 2:] - 2 * p[1:-1, 1:-1] + p[1:-1, :-2]) / dx ** 2
                   + (p[2:, 1:-1] - 2 * p[1:-1, 1:-1] + p[:-2, 1:-1]) / dy ** 2)
            assert rel_l2(lap, rhs.astype(np.float64)) <= 1e-5
    b.close()


def test_tc_and_matrix_engines_agree(monkeypatch):
    """The tcgen05 and mma.sync forms of the same products agree to FP32
    rounding."""
    require_gpu()
    nx, ny = 32, 64
    rhs = inputs.random_field(nx, ny, seed=3)
    a = forced_basin(monkeypatch, nx, ny, 0)
    got41 = to_np(a.poisson_solve(rhs))
    a.close()
    b = forced_basin(monkeypatch, nx, ny, 0, engine=40)
    got40 = to_np(b.poisson_solve(rhs))
    b.close()
    assert rel_l2(got41, got40) <= 1e-6


@pytest.mark.parametrize("nx,ny,levels", [(64, 128, 1), (128, 128, 1), (128, 256, 2),
                                          (64, 64, 0)])
def test_tc_engine_in_the_step(nx, ny, levels, monkeypatch):
    """100 FP32 CGP steps (the restriction's partial planes feed the solve at
    l >= 1) against the oracle's FP64 steps."""
    require_gpu()
    w0 = inputs.perturbation(nx, ny, seed=11) * 50.0
    ref = O.run(w0, O.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=levels, dt=5e-5), 100)
    b = forced_basin(monkeypatch, nx, ny, levels, dt=5e-5)
    b.set_state(w0)
    b.step(100)
    assert rel_l2(to_np(b.state()), ref) <= 1e-4
    b.close()


def test_tc_engine_in_an_ensemble_equals_standalone_handles(monkeypatch):
    """Members on engine 41 (one CTA per member, one launch per group):
    bitwise the stand-alone handles' steps."""
    require_gpu()
    monkeypatch.setenv("QG_SOLVE_ENGINE", str(TC))
    monkeypatch.setenv("QG_FINE_ROWS", "64")   # the members' (batched) tile
    members = [
        dict(nx=32, ny=64, Re=200.0, Ro=0.0016, levels=0, dt=1e-4, amp=1.0),
        dict(nx=64, ny=128, Re=312.5, Ro=0.0025, levels=1, dt=1e-4, amp=1.3),
        dict(nx=128, ny=256, Re=800.0, Ro=0.0016, levels=2, dt=5e-5, amp=0.5),
        dict(nx=128, ny=128, Re=200.0, Ro=0.0016, levels=1, dt=5e-5, amp=1.0),
    ]
    ens = qg.Ensemble(members, dtype="f32")
    solo = [qg.Basin(m["nx"], m["ny"], Re=m["Re"], Ro=m["Ro"], levels=m["levels"], dt=m["dt"],
                     amp=m["amp"], dtype="f32") for m in members]
    for i, m in enumerate(members):
        assert qg.qg_solve_engine(ens.member(i).h) == TC
        assert qg.qg_solve_engine(solo[i].h) == TC
        w = inputs.perturbation(m["nx"], m["ny"], seed=80 + i) * 40.0
        ens.member(i).set_state(w)
        solo[i].set_state(w)
    ens.step(10)
    for b in solo:
        b.step(10)
    ens.synchronize()
    for i, b in enumerate(solo):
        b.synchronize()
        assert np.array_equal(to_np(ens.member(i).state()), to_np(b.state())), i
        b.close()
    ens.close()
