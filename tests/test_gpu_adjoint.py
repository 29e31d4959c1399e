"""GPU parity of the discrete adjoint (qg_tape_*, qg_adjoint_step,
qg_energy_gradient and the autograd wrapper) with the FP64 adjoint oracle,
which is itself pinned to forward differences of the forward oracle."""
import numpy as np
import pytest

from oracle import qg_adjoint as AD
from oracle import qg_oracle as O
from paper_1308_3290_gb300 import adjoint, inputs, qg
from tests.gpu_util import rel_l2, require_gpu, to_np

pytestmark = pytest.mark.gpu


def basin(nx, ny, levels, dtype, dt=1e-4):
    return qg.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=levels, dt=dt, dtype=dtype)


@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_adjoint_step_matches_oracle(levels, dtype, tol):
    torch = require_gpu()
    nx, ny = 64, 128
    w0 = inputs.perturbation(nx, ny, seed=31) * 50.0
    lam0 = inputs.random_field(nx, ny, seed=32)
    b = basin(nx, ny, levels, dtype)
    b.set_state(w0)
    qg.qg_tape_begin(b.h, 1, 1)
    b.step(1)
    td = torch.float64 if dtype == "f64" else torch.float32
    lam = torch.as_tensor(lam0, dtype=td, device="cuda").contiguous()
    g = torch.zeros_like(lam)
    qg.qg_adjoint_step(b.h, 1, lam, g)
    b.synchronize()
    ob = O.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=levels, dt=1e-4)
    ref_lam, ref_g = AD.adjoint_step(O.embed(w0), lam0, ob, O.forcing_one_layer(ob))
    assert rel_l2(to_np(lam), ref_lam) <= tol
    assert rel_l2(to_np(g), ref_g) <= tol
    with pytest.raises(qg.QGError):
        qg.qg_adjoint_step(b.h, 1, lam, g)          # the cursor is at 0
    qg.qg_tape_end(b.h)
    b.close()


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-11), ("f32", 1e-5)])
def test_energy_gradient_matches_oracle(dtype, tol):
    torch = require_gpu()
    nx, ny = 64, 128
    w0 = inputs.perturbation(nx, ny, seed=33) * 50.0
    b = basin(nx, ny, 1, dtype)
    b.set_state(w0)
    qg.qg_tape_begin(b.h, 1, 1)
    td = torch.float64 if dtype == "f64" else torch.float32
    g = torch.zeros((ny - 1, nx - 1), dtype=td, device="cuda")
    qg.qg_energy_gradient(b.h, 2.0, g)
    b.synchronize()
    ob = O.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=1, dt=1e-4)
    assert rel_l2(to_np(g), 2.0 * AD.energy_gradient(O.embed(w0), ob)) <= tol
    b.close()


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-9), ("f32", 1e-3)])
def test_mean_energy_gradient_matches_oracle(dtype, tol):
    """The autograd wrapper's dJ/dF of the time-mean kinetic energy against
    the oracle's; checkpointing every 16 steps gives the result of keeping
    every state to rounding."""
    torch = require_gpu()
    nx, ny, N, first = 64, 128, 60, 40
    w0 = inputs.perturbation(nx, ny, seed=34) * 50.0
    ob = O.Basin(nx, ny, Re=200.0, Ro=0.0016, levels=1, dt=1e-4)
    F0 = inputs.perturbed_forcing_field(nx, ny, seed=5, Ro=0.0016)
    J_ref, g_ref = AD.mean_energy_gradient(w0, ob, F0, N, first)
    td = torch.float64 if dtype == "f64" else torch.float32
    grads = []
    for every in (1, 16):
        b = basin(nx, ny, 1, dtype)
        F = torch.as_tensor(F0, dtype=td, device="cuda").contiguous().requires_grad_(True)
        J = adjoint.mean_kinetic_energy(F, b, torch.as_tensor(w0, dtype=td, device="cuda"),
                                        N, first, every)
        J.backward()
        assert float(J.detach()) == pytest.approx(J_ref, rel=1e-10 if dtype == "f64" else 1e-5)
        grads.append(to_np(F.grad))
        b.close()
    assert rel_l2(grads[0], g_ref) <= tol
    # the recomputed segments start from a fresh restriction of the
    # checkpoint instead of the previous step's partial sums: equal to rounding
    assert rel_l2(grads[1], grads[0]) <= (1e-11 if dtype == "f64" else 1e-5)
