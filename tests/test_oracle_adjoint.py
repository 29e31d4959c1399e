"""Pins of the FP64 adjoint oracle (oracle/qg_adjoint.py) to things other
than itself: the forward oracle's own finite differences (exact for the
quadratic right-hand side), dot-product identities of each transposed
operator, and central-difference gradients of the time-mean energy."""
import numpy as np
import pytest

from oracle import qg_adjoint as AD
from oracle import qg_oracle as O
from paper_1308_3290_gb300 import inputs


def rnd(nx, ny, seed, scale=1.0):
    return O.embed(inputs.random_field(nx, ny, seed) * scale)


@pytest.mark.parametrize("nx,ny", [(16, 32), (32, 16)])
def test_arakawa_operators_are_skew(nx, ny):
    """Sum a J(p, c) = -Sum c J(p, a) and Sum a J(c, y) = -Sum c J(a, y) for
    fields that vanish on the walls."""
    b = O.Basin(nx, ny)
    p, a, c = rnd(nx, ny, 1), rnd(nx, ny, 2), rnd(nx, ny, 3)
    lhs = np.sum(O.interior(a) * O.arakawa(p, c, b.dx, b.dy))
    rhs = -np.sum(O.interior(c) * O.arakawa(p, a, b.dx, b.dy))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)
    lhs = np.sum(O.interior(a) * AD.beta_jacobian(c, b))
    rhs = -np.sum(O.interior(c) * AD.beta_jacobian(a, b))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


@pytest.mark.parametrize("levels", [0, 1, 2])
def test_projection_is_self_adjoint(levels):
    b = O.Basin(32, 64, levels=levels)
    u, v = rnd(32, 64, 4), rnd(32, 64, 5)
    lhs = np.sum(O.interior(O.cgp_psi(u, b)) * O.interior(v))
    rhs = np.sum(O.interior(u) * O.interior(O.cgp_psi(v, b)))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


@pytest.mark.parametrize("levels", [0, 1, 2])
def test_rhs_adjoint_against_forward_differences(levels):
    """G is quadratic in w, so the central difference of the forward oracle's
    cgp_rhs is its exact directional derivative."""
    b = O.Basin(32, 64, levels=levels)
    w, dw, lam = rnd(32, 64, 6, 20.0), rnd(32, 64, 7), rnd(32, 64, 8)
    eps = 1e-3
    dG = (O.cgp_rhs(w + eps * dw, b) - O.cgp_rhs(w - eps * dw, b)) / (2 * eps)
    lhs = np.sum(dG * O.interior(lam))
    rhs = np.sum(O.interior(dw) * AD.rhs_adjoint(lam, w, O.cgp_psi(w, b), b))
    assert abs(lhs - rhs) <= 1e-9 * np.sqrt(np.sum(dG ** 2) * np.sum(lam ** 2))


@pytest.mark.parametrize("levels", [0, 1])
def test_adjoint_step_against_forward_differences(levels):
    b = O.Basin(32, 64, levels=levels, dt=1e-4)
    w = rnd(32, 64, 9, 50.0)
    dw = rnd(32, 64, 10)
    lam = inputs.random_field(32, 64, 11)
    F = O.forcing_one_layer(b)
    dF = inputs.random_field(32, 64, 12) * np.abs(F).max()
    lam_n, gF = AD.adjoint_step(w, lam, b, F)
    from dataclasses import replace

    def step(wv, Fv):
        return O.interior(O.cgprk3_step(wv, replace(b, forcing=Fv)))

    eps = 1e-4
    d = (step(w + eps * dw, F) - step(w - eps * dw, F)) / (2 * eps)
    lhs, rhs = np.sum(d * lam), np.sum(O.interior(dw) * lam_n)
    assert abs(lhs - rhs) <= 1e-8 * abs(lhs)
    eps = 1e-2     # F moves w by O(dt eps |dF|): larger steps keep rounding out
    d = (step(w, F + eps * dF) - step(w, F - eps * dF)) / (2 * eps)
    lhs, rhs = np.sum(d * lam), np.sum(dF * gF)
    assert abs(lhs - rhs) <= 1e-8 * abs(lhs)


def test_energy_gradient_against_differences():
    """E(A w) is quadratic in w: central differences are exact."""
    b = O.Basin(32, 64, levels=1)
    w, dw = rnd(32, 64, 13, 20.0), rnd(32, 64, 14)
    eps = 1e-3
    d = (AD.energy(w + eps * dw, b) - AD.energy(w - eps * dw, b)) / (2 * eps)
    g = np.sum(O.interior(dw) * AD.energy_gradient(w, b))
    assert abs(d - g) <= 1e-9 * abs(d)


def test_mean_energy_gradient_central_differences():
    """dJ/dF against central differences of the forward oracle along seeded
    unit directions, and the Taylor remainder is second order."""
    nx, ny, N, first = 16, 32, 24, 12
    b = O.Basin(nx, ny, levels=1, dt=2e-4)
    w0 = inputs.perturbation(nx, ny, seed=15) * 100.0
    F = O.forcing_one_layer(b)
    J, g = AD.mean_energy_gradient(w0, b, F, N, first)
    assert J == pytest.approx(AD.mean_energy(w0, b, F, N, first), rel=1e-13)
    rng = np.random.default_rng(16)
    for _ in range(4):
        d = rng.normal(size=F.shape)
        d /= np.linalg.norm(d)
        h = 1e-6 * np.abs(F).max()
        fd = (AD.mean_energy(w0, b, F + h * d, N, first)
              - AD.mean_energy(w0, b, F - h * d, N, first)) / (2 * h)
        assert np.sum(g * d) == pytest.approx(fd, rel=1e-6)
    d = rng.normal(size=F.shape)
    h1 = 1e-1 * np.abs(F).max() / np.linalg.norm(d)
    r = []
    for h in (h1, h1 / 2):
        r.append(abs(AD.mean_energy(w0, b, F + h * d, N, first) - J - h * np.sum(g * d)))
    assert 3.0 < r[0] / r[1] < 5.0
