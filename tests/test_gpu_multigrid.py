"""The multigrid solver of the CGP step (Section 3: CGP is independent of the
Poisson solver on the coarse grid; the paper names the V-cycle multigrid).

Its result approaches the discrete solution, which the oracle computes
exactly (Section 4.3's sine transforms), by a fixed factor per V-cycle; the
CGP step with multigrid solves follows the oracle's step to within what the
cycles leave."""
import numpy as np
import pytest

from oracle import qg_oracle as O
from paper_1308_3290_gb300 import inputs, qg
from tests.gpu_util import rel_l2, require_gpu, to_np

pytestmark = pytest.mark.gpu


def solve_err(nx, ny, dtype, cycles, seed):
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=0, dt=1e-4, dtype=dtype)
    qg.qg_set_solver(b.h, qg.QG_SOLVER_MULTIGRID, cycles)
    rhs = inputs.random_field(nx, ny, seed=seed)
    got = to_np(b.poisson_solve(rhs))
    b.close()
    ref = O.poisson_solve(rhs, nx, ny, 1.0 / nx, 2.0 / ny)
    return rel_l2(got, ref)


@pytest.mark.parametrize("nx,ny,rate", [(64, 128, 5.0), (32, 128, 2.5), (512, 1024, 5.0),
                                        (128, 128, 2.5), (64, 256, 2.5)])
def test_vcycles_converge_to_the_discrete_solution(nx, ny, rate):
    """Each V(2,2) cycle cuts the error against the exact discrete solution
    by at least `rate` (equal spacings: 5x; spacings a factor 2 apart:
    2.5x); 30 cycles in FP64 reach 1e-11."""
    require_gpu()
    errs = [solve_err(nx, ny, "f64", c, seed=nx + ny) for c in (1, 2, 3, 4)]
    for a, b in zip(errs, errs[1:]):
        assert b <= a / rate, errs
    assert solve_err(nx, ny, "f64", 30, seed=nx + ny) <= 1e-11


def test_fp32_multigrid_reaches_rounding():
    require_gpu()
    assert solve_err(512, 1024, "f32", 12, seed=3) <= 1e-5


@pytest.mark.parametrize("levels,cycles,tol", [(0, 3, 1e-6), (1, 3, 1e-6), (2, 3, 1e-6)])
def test_cgp_step_with_multigrid_follows_the_oracle(levels, cycles, tol):
    """100 FP64 steps with warm-started V-cycles against the oracle's steps
    with exact solves."""
    require_gpu()
    nx, ny = 64, 128
    w0 = inputs.perturbation(nx, ny, seed=8) * 50.0
    ob = O.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=levels, dt=1e-4)
    ref = O.run(w0, ob, 100)
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=levels, dt=1e-4, dtype="f64")
    qg.qg_set_solver(b.h, qg.QG_SOLVER_MULTIGRID, cycles)
    b.set_state(w0)
    b.step(100)
    got = to_np(b.state())
    assert rel_l2(got, ref) <= tol, rel_l2(got, ref)
    # more cycles: closer
    qg.qg_set_solver(b.h, qg.QG_SOLVER_MULTIGRID, 12)
    b.set_state(w0)
    b.step(100)
    assert rel_l2(to_np(b.state()), ref) <= 1e-11
    # and back to the sine transforms: the exact step again
    qg.qg_set_solver(b.h, qg.QG_SOLVER_FFT, 0)
    b.set_state(w0)
    b.step(100)
    assert rel_l2(to_np(b.state()), ref) <= 1e-12
    b.close()


def test_multigrid_step_is_deterministic():
    require_gpu()
    nx, ny = 256, 512
    w0 = inputs.perturbation(nx, ny, seed=9) * 30.0
    outs = []
    for _ in range(2):
        b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=2, dt=2e-5, dtype="f32")
        qg.qg_set_solver(b.h, qg.QG_SOLVER_MULTIGRID, 3)
        b.set_state(w0)
        b.step(20)
        outs.append(to_np(b.state()))
        b.close()
    assert np.array_equal(outs[0], outs[1])


def test_multigrid_unsupported_cases():
    require_gpu()
    # two layers
    b = qg.Basin(64, 64, Re=2.49e-4 / 3.57e-7, Ro=2.49e-4, Fr=0.087, delta=0.2, sigma=1.43e-3,
                 levels=1, dt=1e-4, dtype="f64", layers=2, y0=-0.5, y1=0.5)
    with pytest.raises(qg.QGError) as e:
        qg.qg_set_solver(b.h, qg.QG_SOLVER_MULTIGRID, 4)
    assert e.value.status == qg.QG_ERR_UNSUPPORTED
    b.close()
    # sides more than a factor 4 apart
    b = qg.Basin(16, 256, Re=200.0, Ro=0.0016, levels=0, dt=1e-4, dtype="f64")
    with pytest.raises(qg.QGError) as e:
        qg.qg_set_solver(b.h, qg.QG_SOLVER_MULTIGRID, 4)
    assert e.value.status == qg.QG_ERR_UNSUPPORTED
    b.close()
    # cycles out of range; the adjoint needs the exact solve
    b = qg.Basin(64, 128, Re=200.0, Ro=0.0016, levels=1, dt=1e-4, dtype="f64")
    with pytest.raises(qg.QGError) as e:
        qg.qg_set_solver(b.h, qg.QG_SOLVER_MULTIGRID, 0)
    assert e.value.status == qg.QG_ERR_ARG
    qg.qg_set_solver(b.h, qg.QG_SOLVER_MULTIGRID, 4)
    with pytest.raises(qg.QGError) as e:
        qg.qg_tape_begin(b.h, 1, 10)
    assert e.value.status == qg.QG_ERR_UNSUPPORTED
    b.close()


def test_multigrid_with_adaptive_step_and_time_mean():
    """The solver switch composes with the adaptive step (Eq. dt) and the
    time-mean statistics: 12 warm-started cycles per solve follow the
    oracle's exact-solve trajectory, step sizes and mean psi."""
    torch = require_gpu()
    nx, ny, n, c = 64, 128, 30, 0.3
    w0 = inputs.perturbation(nx, ny, seed=3) * 50.0
    ob = O.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=1, dt=1e-3)
    ref, dts = O.run_adaptive(w0, ob, n, c)
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=1, dt=1e-3, dtype="f64")
    qg.qg_set_solver(b.h, qg.QG_SOLVER_MULTIGRID, 12)
    qg.qg_set_cfl(b.h, c)
    b.set_state(w0)
    b.step(n)
    assert rel_l2(to_np(b.state()), ref) <= 1e-9
    t, dt_last = qg.qg_get_time(b.h)
    assert t == pytest.approx(sum(dts), rel=1e-9)
    assert dt_last == pytest.approx(dts[-1], rel=1e-9)
    b.close()

    ob = O.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=2, dt=1e-4)
    ref = O.mean_psi(w0, ob, 5, 25)
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=2, dt=1e-4, dtype="f64")
    qg.qg_set_solver(b.h, qg.QG_SOLVER_MULTIGRID, 12)
    b.set_state(w0)
    b.step(5)
    qg.qg_stats_begin(b.h)
    b.step(20)
    out = torch.empty((ny - 1, nx - 1), dtype=torch.float64, device="cuda")
    assert qg.qg_stats_mean_psi(b.h, out) == 20
    b.synchronize()
    assert rel_l2(to_np(out), ref) <= 1e-9
    b.close()


def test_multigrid_on_an_ensemble_member_equals_a_standalone_handle(monkeypatch):
    """The solver switch on one member of an ensemble: its steps are bitwise
    those of a stand-alone handle with the same switch (the V-cycles do not
    depend on how the member's graph is launched); the other members keep
    the sine transforms and follow the oracle."""
    require_gpu()
    monkeypatch.setenv("QG_FINE_ROWS", "64")   # the members' (batched) tile
    members = [dict(nx=64, ny=128, Re=200.0, Ro=0.0016, levels=1, dt=1e-4),
               dict(nx=128, ny=256, Re=200.0, Ro=0.0016, levels=2, dt=5e-5)]
    w = [inputs.perturbation(m["nx"], m["ny"], seed=60 + i) * 40.0 for i, m in enumerate(members)]
    ens = qg.Ensemble(members, dtype="f32")
    qg.qg_set_solver(ens.member(1).h, qg.QG_SOLVER_MULTIGRID, 3)
    for i in range(2):
        ens.member(i).set_state(w[i])
    ens.step(15)
    ens.synchronize()
    m = members[1]
    solo = qg.Basin(m["nx"], m["ny"], Re=m["Re"], Ro=m["Ro"], levels=m["levels"], dt=m["dt"],
                    dtype="f32")
    qg.qg_set_solver(solo.h, qg.QG_SOLVER_MULTIGRID, 3)
    solo.set_state(w[1])
    solo.step(15)
    assert np.array_equal(to_np(ens.member(1).state()), to_np(solo.state()))
    m0 = members[0]
    ref = O.run(w[0], O.Basin(m0["nx"], m0["ny"], Re=200.0, Ro=0.0016, levels=1, dt=1e-4), 15)
    assert rel_l2(to_np(ens.member(0).state()), ref) <= 1e-5
    solo.close()
    ens.close()
