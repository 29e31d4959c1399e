"""GPU parity of the two-layer CGPRK3 step (Section 2.2, Table 2 Experiment 1
parameters) with the oracle."""
import numpy as np
import pytest

from oracle import qg_oracle as O
from paper_1308_3290_gb300 import inputs, qg
from tests.gpu_util import assert_fields_close, rel_l2, require_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-11), ("f32", 1e-4)])
@pytest.mark.parametrize("levels", [0, 1])
@pytest.mark.parametrize("nx,ny", [(64, 64), (64, 128)])
def test_two_layer_steps(dtype, tol, levels, nx, ny):
    """The square basin on N x N and on N x 2N intervals (dy = dx/2)."""
    require_gpu()
    p = dict(Ro=2.49e-4, Fr=0.087, delta=0.2, sigma=1.43e-3)
    A = 3.57e-7
    Re = p["Ro"] / A
    Q1 = inputs.smooth_field(nx, ny, seed=1, amp=0.05, noise=0.01)
    Q2 = inputs.smooth_field(nx, ny, seed=2, amp=0.02, noise=0.01)
    ob = O.TwoLayer(nx, ny, A=A, levels=levels, dt=1e-4, **p)
    a1, a2 = O.embed(Q1), O.embed(Q2)
    for _ in range(50):
        a1, a2 = O.cgprk3_step_two_layer(a1, a2, ob)
    b = qg.Basin(nx, ny, Re=Re, levels=levels, dt=1e-4, dtype=dtype, layers=2,
                 y0=-0.5, y1=0.5, **p)
    b.set_state(Q1, 0)
    b.synchronize()
    b.set_state(Q2, 1)
    b.step(50)
    g1, g2 = to_np(b.state(0)), to_np(b.state(1))
    assert_fields_close(g1, O.interior(a1), tol)
    assert_fields_close(g2, O.interior(a2), tol)
    b.close()


def test_two_layer_full_size_one_step():
    """One step of the two-layer 1024 x 2048, l = 1, FP32 workload the
    benchmark times (Table 2 Experiment 1), against one FP64 oracle step."""
    require_gpu()
    nx, ny = 1024, 2048
    p = dict(Ro=2.49e-4, Fr=0.087, delta=0.2, sigma=1.43e-3)
    A = 3.57e-7
    Q1 = inputs.smooth_field(nx, ny, seed=3, amp=0.05, noise=0.01)
    Q2 = inputs.smooth_field(nx, ny, seed=4, amp=0.02, noise=0.01)
    ob = O.TwoLayer(nx, ny, A=A, levels=1, dt=1e-5, **p)
    a1, a2 = O.cgprk3_step_two_layer(O.embed(Q1), O.embed(Q2), ob)
    b = qg.Basin(nx, ny, Re=p["Ro"] / A, levels=1, dt=1e-5, dtype="f32", layers=2,
                 y0=-0.5, y1=0.5, **p)
    b.set_state(Q1, 0)
    b.synchronize()
    b.set_state(Q2, 1)
    b.step(1)
    for layer, q0, ref in ((0, Q1, O.interior(a1)), (1, Q2, O.interior(a2))):
        got = to_np(b.state(layer))
        assert_fields_close(got, ref, 1e-6, max_tol=64 * 2.0 ** -24)
        assert_fields_close(got - q0, ref - q0, 1e-3, max_tol=1.0)
        assert np.abs((got - q0) - (ref - q0)).max() <= 64 * 2.0 ** -24 * np.abs(q0).max()
    b.close()
