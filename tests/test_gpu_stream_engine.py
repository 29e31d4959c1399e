"""Engine 50 of the elliptic solve (solve_stream.cu: radix-16 passes with
the values in registers, one CTA per sequence pair, three launches) against
the oracle's sine-transform solve of Section 4.3 (Eqs. ffft-1, ialpha,
ifft-1): every length it takes (FFT lengths 512 to 16384, with radix-2, 4
and 8 remainder passes and none; 1, 2 and 4 sequence pairs per CTA), one
and two layers, FP64 and FP32, element-wise; the exact discrete
eigenmodes; and the whole step."""
import numpy as np
import pytest

from oracle import qg_oracle as O
from paper_1308_3290_gb300 import inputs, qg
from tests.gpu_util import assert_fields_close, rel_l2, require_gpu, to_np
from tests.test_gpu_edges import eigenvalue, lap_h, mode

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6}
# per element, relative to the field's largest value
MAX = {"f64": 1e-12, "f32": 64 * 2.0 ** -24}


def basin(nx, ny, dtype, levels=0, dt=1e-4, **kw):
    b = qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=levels, dt=dt, dtype=dtype, **kw)
    assert qg.qg_solve_engine(b.h) == 50
    return b


@pytest.fixture(autouse=True)
def _force_engine(monkeypatch):
    monkeypatch.setenv("QG_SOLVE_ENGINE", "50")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny", [
    (256, 512), (512, 256), (512, 1024), (1024, 512), (2048, 512), (512, 4096),
    (2048, 4096),
])
def test_poisson_parity(dtype, nx, ny):
    """FFT lengths 2N = 512 (remainder radix 2), 1024 (4), 2048 (8), 4096
    (none), 8192 (2); the 2048 x 4096 full grid is the l = 0 workload."""
    require_gpu()
    b = basin(nx, ny, dtype)
    rhs = inputs.smooth_field(nx, ny, seed=nx + 3 * ny, noise=0.3)
    got = to_np(b.poisson_solve(rhs))
    ref = O.poisson_solve(rhs, nx, ny, 1.0 / nx, 2.0 / ny)
    assert_fields_close(got, ref, TOL[dtype], MAX[dtype])
    b.close()


@pytest.mark.parametrize("nx,ny", [(8192, 512), (512, 8192)])
def test_longest_fp32_sequences(nx, ny):
    """FFT length 16384 (CTAs of 1024 threads), FP32 only."""
    require_gpu()
    b = basin(nx, ny, "f32")
    rhs = inputs.random_field(nx, ny, seed=11)
    got = to_np(b.poisson_solve(rhs))
    ref = O.poisson_solve(rhs, nx, ny, 1.0 / nx, 2.0 / ny)
    assert rel_l2(got, ref) <= TOL["f32"]
    b.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_white_noise_and_eigenmodes(dtype):
    """A white-noise right-hand side (every mode excited), and the discrete
    eigenmodes: the lowest by its forward error, two higher ones by the
    residual of the 5-point operator (see test_gpu_edges)."""
    require_gpu()
    nx, ny = 1024, 2048
    dx, dy = 1.0 / nx, 2.0 / ny
    b = basin(nx, ny, dtype)
    rhs = inputs.random_field(nx, ny, seed=5)
    got = to_np(b.poisson_solve(rhs))
    assert rel_l2(got, O.poisson_solve(rhs, nx, ny, dx, dy)) <= TOL[dtype]
    for n, (k, l) in enumerate(((1, 2), (nx // 3, ny // 5), (nx - 3, ny - 5))):
        want = mode(nx, ny, k, l)
        rhs = eigenvalue(nx, ny, dx, dy, k, l) * want
        got = to_np(b.poisson_solve(rhs))
        if n == 0:
            assert rel_l2(got, want) <= TOL[dtype], (k, l)
        else:
            rhs_t = rhs.astype(np.float32 if dtype == "f32" else np.float64)
            res = rel_l2(lap_h(got, dx, dy), rhs_t.astype(np.float64))
            assert res <= (1e-5 if dtype == "f32" else 1e-13), (k, l, res)
    b.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_two_layer_solve(dtype):
    """The coupled solve of Eqs. isub-1/2 in the y pass (both layers of one
    x-mode share a transform)."""
    require_gpu()
    nx, ny = 512, 1024
    p = dict(Ro=2.49e-4, Fr=0.087, delta=0.2, sigma=1.43e-3)
    b = qg.Basin(nx, ny, Re=697.16, levels=0, dt=1e-5, dtype=dtype, layers=2, y0=-0.5,
                 y1=0.5, **p)
    assert qg.qg_solve_engine(b.h) == 50
    Q1 = inputs.smooth_field(nx, ny, seed=1, noise=0.1)
    Q2 = inputs.smooth_field(nx, ny, seed=2, noise=0.1)
    got = to_np(b.poisson_solve(np.stack([Q1, Q2])))
    r1, r2 = O.elliptic_two_layer(Q1, Q2, nx, ny, 1 / nx, 1 / ny, p["Ro"], p["Fr"], p["delta"])
    assert rel_l2(got[0], r1) <= TOL[dtype] * 5
    assert rel_l2(got[1], r2) <= TOL[dtype] * 5
    b.close()


def test_fp64_step_matches_oracle():
    """FP64 CGPRK3 steps against the oracle: 20 of a 512 x 1024 basin at
    l = 0 and 8 of a 1024 x 2048 one at l = 1 (elliptic grid 512 x 1024)."""
    require_gpu()
    for nx, ny, lv, n in ((512, 1024, 0, 20), (1024, 2048, 1, 8)):
        w0 = inputs.perturbation(nx, ny, seed=3) * 50.0
        ref = O.run(w0, O.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=lv, dt=1e-5), n)
        b = basin(nx, ny, "f64", levels=lv, dt=1e-5)
        b.set_state(w0)
        b.step(n)
        assert rel_l2(to_np(b.state()), ref) <= 1e-12
        b.close()


def test_launch_count(monkeypatch):
    """Three solve launches per stage instead of one."""
    require_gpu()
    b = basin(512, 1024, "f32")
    n50 = qg.qg_step_kernel_count(b.h)
    b.close()
    monkeypatch.setenv("QG_SOLVE_ENGINE", "33")
    b = qg.Basin(512, 1024, Re=200.0, Ro=0.0016, levels=0, dt=1e-4, dtype="f32")
    assert qg.qg_solve_engine(b.h) == 33
    assert n50 == qg.qg_step_kernel_count(b.h) + 6
    b.close()


def test_batched_in_an_ensemble_equals_standalone_handles(monkeypatch):
    """Ensemble groups solve with engine 50 as one batch (a work queue over
    the three passes of every member in one launch when the y length is
    twice the x length, else three launches with the members' CTAs side by
    side): bitwise the states of stand-alone handles with the same engine.
    The first and third members share an elliptic grid (256 x 512, spacing
    1/256) at different levels."""
    require_gpu()
    from tests.test_gpu_ensemble import _groups
    monkeypatch.setenv("QG_FINE_ROWS", "64")   # the members' (batched) tile
    members = [
        dict(nx=512, ny=1024, Re=200.0, Ro=0.0016, levels=1, dt=2e-5, amp=1.0),
        dict(nx=1024, ny=512, Re=450.0, Ro=0.0036, levels=1, dt=2e-5, amp=0.7),
        dict(nx=1024, ny=2048, Re=312.5, Ro=0.0025, levels=2, dt=1e-5, amp=1.3),
        dict(nx=512, ny=512, Re=800.0, Ro=0.0016, levels=0, dt=1e-5, amp=0.5),
    ]
    ens = qg.Ensemble(members, dtype="f32")
    solo = [qg.Basin(m["nx"], m["ny"], Re=m["Re"], Ro=m["Ro"], levels=m["levels"], dt=m["dt"],
                     amp=m["amp"], dtype="f32") for m in members]
    for b in solo:
        assert qg.qg_solve_engine(b.h) == 50
    for i, m in enumerate(members):
        w = inputs.perturbation(m["nx"], m["ny"], seed=60 + i) * 50.0
        ens.member(i).set_state(w)
        solo[i].set_state(w)
    ens.step(4)
    for b in solo:
        b.step(4)
    ens.synchronize()
    for i, b in enumerate(solo):
        b.synchronize()
        assert np.array_equal(to_np(ens.member(i).state()), to_np(b.state())), i
        b.close()
    n_solve, n_fine = _groups(members)
    assert n_solve == 3
    # the 256 x 512 group (y length twice the x length) solves as one
    # work-queue launch, the 512 x 256 and 512 x 512 groups as three
    assert ens.kernel_count() == 3 * (1 + 3 + 3 + n_fine)
    ens.close()
