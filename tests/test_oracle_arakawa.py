"""Pins of the oracle's Arakawa Jacobian (Section 4.1, Eqs. ja1, j1-j3) and
of the fine-grid right-hand side.

Discrete conservation (sum psi J = sum w J = 0 with zero walls, sum J = 0 for
compactly supported fields), skew-symmetry, the closed form of J(psi, y), and
second-order consistency of each of J1, J2, J3 against the analytic Jacobian.
"""
import numpy as np
import pytest

from oracle import qg_oracle as O


def zero_wall_field(nx, ny, seed, ring=0):
    rng = np.random.default_rng(seed)
    a = np.zeros((ny + 1, nx + 1))
    a[1 + ring:ny - ring, 1 + ring:nx - ring] = rng.normal(size=(ny - 1 - 2 * ring, nx - 1 - 2 * ring))
    return a


@pytest.mark.parametrize("nx,ny,dx,dy", [(16, 32, 1 / 16, 1 / 16), (32, 32, 1 / 32, 1 / 64)])
def test_energy_and_enstrophy_conservation(nx, ny, dx, dy):
    psi = zero_wall_field(nx, ny, 1)
    w = zero_wall_field(nx, ny, 2)
    J = O.arakawa(psi, w, dx, dy)
    scale = np.sum(np.abs(J)) * max(np.abs(psi).max(), np.abs(w).max())
    assert abs(np.sum(O.interior(psi) * J)) < 1e-14 * scale
    assert abs(np.sum(O.interior(w) * J)) < 1e-14 * scale


def test_sum_of_jacobian_vanishes_for_compact_support():
    nx, ny = 16, 32
    psi = zero_wall_field(nx, ny, 3, ring=1)
    w = zero_wall_field(nx, ny, 4, ring=1)
    J = O.arakawa(psi, w, 1 / 16, 1 / 16)
    assert abs(np.sum(J)) < 1e-13 * np.sum(np.abs(J))


def test_sum_of_jacobian_does_not_vanish_with_only_zero_walls():
    """With psi = w = 0 on the walls alone, sum J is not a conserved
    quantity (this is why the conservation pins above use compact support)."""
    nx, ny = 16, 32
    J = O.arakawa(zero_wall_field(nx, ny, 5), zero_wall_field(nx, ny, 6), 1 / 16, 1 / 16)
    assert abs(np.sum(J)) > 1e-3 * np.sum(np.abs(J))


def test_skew_symmetry():
    rng = np.random.default_rng(7)
    a = rng.normal(size=(17, 9))
    b = rng.normal(size=(17, 9))
    assert np.allclose(O.arakawa(a, b, 0.1, 0.2), -O.arakawa(b, a, 0.1, 0.2), rtol=0, atol=1e-12)
    assert np.allclose(O.arakawa(a, a, 0.1, 0.2), 0.0, atol=1e-12)


def test_beta_term_closed_form():
    """J(psi, y) = (4 c_j + c_{j+1} + c_{j-1})/6 with
    c_j = (psi_{i+1,j} - psi_{i-1,j})/(2 dx): J1 and J3 each give c_j and J2
    gives (c_{j+1} + c_{j-1})/2 when q = y."""
    nx, ny = 16, 32
    dx, dy = 1 / 16, 2 / 32
    psi = np.random.default_rng(9).normal(size=(ny + 1, nx + 1))
    y = -1.0 + dy * np.arange(ny + 1)
    Y = np.repeat(y[:, None], nx + 1, axis=1)
    c = (psi[:, 2:] - psi[:, :-2]) / (2 * dx)           # c[j, i-1]
    want = (4 * c[1:-1] + c[2:] + c[:-2]) / 6.0
    assert np.allclose(O.arakawa(psi, Y, dx, dy), want, rtol=0, atol=1e-11)


def _analytic_fields(nx, ny):
    x = np.arange(nx + 1) / nx
    y = -1.0 + 2.0 * np.arange(ny + 1) / ny
    X, Y = np.meshgrid(x, y)
    psi = np.sin(np.pi * X) * np.cos(0.5 * np.pi * Y) + 0.3 * X * Y
    q = np.cos(1.3 * X) * np.sin(np.pi * Y) + X ** 2
    psi_x = np.pi * np.cos(np.pi * X) * np.cos(0.5 * np.pi * Y) + 0.3 * Y
    psi_y = -0.5 * np.pi * np.sin(np.pi * X) * np.sin(0.5 * np.pi * Y) + 0.3 * X
    q_x = -1.3 * np.sin(1.3 * X) * np.sin(np.pi * Y) + 2 * X
    q_y = np.pi * np.cos(1.3 * X) * np.cos(np.pi * Y)
    J = psi_x * q_y - psi_y * q_x                       # Eq. jac (continuous)
    return psi, q, J[1:-1, 1:-1], 1.0 / nx, 2.0 / ny


@pytest.mark.parametrize("which", [0, 1, 2, 3])
def test_second_order_consistency(which):
    errs = []
    for nx in (16, 32, 64, 128):
        psi, q, J, dx, dy = _analytic_fields(nx, 2 * nx)
        terms = O.arakawa_terms(psi, q, dx, dy)
        got = O.arakawa(psi, q, dx, dy) if which == 3 else terms[which]
        errs.append(np.max(np.abs(got - J)))
    ratios = [errs[n] / errs[n + 1] for n in range(3)]
    assert all(3.6 < r < 4.4 for r in ratios), ratios


def test_laplacian5_second_order():
    errs = []
    for nx in (16, 32, 64):
        x = np.arange(nx + 1) / nx
        y = np.arange(2 * nx + 1) / nx
        X, Y = np.meshgrid(x, y)
        f = np.sin(2 * X) * np.exp(Y)
        lap = (-4 + 1) * f
        errs.append(np.max(np.abs(O.laplacian5(f, 1 / nx, 1 / nx) - lap[1:-1, 1:-1])))
    assert 3.8 < errs[0] / errs[1] < 4.2 and 3.8 < errs[1] / errs[2] < 4.2


def test_rhs_energy_budget():
    """At l = 0 the Arakawa terms exchange no energy: dx dy sum psi G equals
    dx dy sum psi ((1/Re) lap w + F) for any state, so a wrong sign or a
    missing Jacobian term shows up here."""
    b = O.Basin(32, 64, Re=200.0, Ro=0.0016, levels=0)
    w = zero_wall_field(32, 64, 12) * 50.0
    psi = O.cgp_psi(w, b)
    G = O.rhs_omega(w, psi, b)
    lhs = np.sum(O.interior(psi) * G)
    rhs = np.sum(O.interior(psi) * (O.laplacian5(w, b.dx, b.dy) / b.Re + O.forcing_one_layer(b)))
    assert abs(lhs - rhs) < 1e-11 * np.sum(np.abs(O.interior(psi) * G))


def test_rhs_enstrophy_budget():
    """sum w J(psi, w) = 0, so dx dy sum w G = sum w (-(1/Ro) J(psi,y) +
    (1/Re) lap w + F)."""
    b = O.Basin(32, 64, Re=200.0, Ro=0.0016, levels=1)
    w = zero_wall_field(32, 64, 13) * 50.0
    psi = O.cgp_psi(w, b)
    G = O.rhs_omega(w, psi, b)
    Y = np.repeat(O.grid_y(b)[:, None], b.nx + 1, axis=1)
    rest = (-O.arakawa(psi, Y, b.dx, b.dy) / b.Ro + O.laplacian5(w, b.dx, b.dy) / b.Re
            + O.forcing_one_layer(b))
    wi = O.interior(w)
    assert abs(np.sum(wi * G) - np.sum(wi * rest)) < 1e-11 * np.sum(np.abs(wi * G))
