"""Pins of the oracle's two-layer model (Section 2.2, Eqs. sub-pr, isub-1/2).

The coupled spectral solve is checked against a dense block solve of Eq.
sub-pr and against the barotropic/baroclinic modal split it is algebraically
equal to; the right-hand side against the layer-wise energy exchange that the
Arakawa scheme forbids.
"""
import numpy as np
import pytest

from oracle import qg_oracle as O
from tests.oracle_helpers import dense_laplacian


@pytest.mark.parametrize("nx,ny,y0,y1", [(8, 16, -1.0, 1.0), (16, 16, -0.5, 0.5)])
def test_coupled_solve_matches_dense_block_solve(nx, ny, y0, y1):
    Ro, Fr, d = 2.49e-4, 0.087, 0.2
    dx, dy = 1.0 / nx, (y1 - y0) / ny
    rng = np.random.default_rng(21)
    Q1 = rng.normal(size=(ny - 1, nx - 1))
    Q2 = rng.normal(size=(ny - 1, nx - 1))
    Lm = Ro * dense_laplacian(nx, ny, dx, dy)
    I = np.eye(Lm.shape[0])
    a, b = Fr / d, Fr / (1 - d)
    M = np.block([[Lm - a * I, a * I], [b * I, Lm - b * I]])
    sol = np.linalg.solve(M, np.concatenate([Q1.ravel(), Q2.ravel()]))
    p1, p2 = O.elliptic_two_layer(Q1, Q2, nx, ny, dx, dy, Ro, Fr, d)
    n = Lm.shape[0]
    assert np.linalg.norm(p1.ravel() - sol[:n]) <= 1e-12 * np.linalg.norm(sol)
    assert np.linalg.norm(p2.ravel() - sol[n:]) <= 1e-12 * np.linalg.norm(sol)


def test_modal_split():
    """psi_bt = delta psi_1 + (1-delta) psi_2 solves Ro lap psi_bt =
    delta Q_1 + (1-delta) Q_2, and psi_bc = psi_1 - psi_2 solves
    (Ro lap - Fr/(delta(1-delta))) psi_bc = Q_1 - Q_2."""
    nx, ny = 32, 32
    dx, dy = 1 / 32, 1 / 32
    Ro, Fr, d = 2.49e-4, 0.087, 0.2
    rng = np.random.default_rng(22)
    Q1 = rng.normal(size=(ny - 1, nx - 1))
    Q2 = rng.normal(size=(ny - 1, nx - 1))
    p1, p2 = O.elliptic_two_layer(Q1, Q2, nx, ny, dx, dy, Ro, Fr, d)
    bt = O.elliptic_one_layer(d * Q1 + (1 - d) * Q2, nx, ny, dx, dy, Ro)
    assert np.linalg.norm(d * p1 + (1 - d) * p2 - bt) <= 1e-12 * np.linalg.norm(bt)
    H = Ro * dense_laplacian(nx, ny, dx, dy) - Fr / (d * (1 - d)) * np.eye((nx - 1) * (ny - 1))
    bc = np.linalg.solve(H, (Q1 - Q2).ravel()).reshape(Q1.shape)
    assert np.linalg.norm(p1 - p2 - bc) <= 1e-11 * np.linalg.norm(bc)


def test_two_layer_rhs_jacobian_terms_conserve_energy_per_layer():
    """With l = 0 and the forcing, viscosity and drag switched off, the
    Arakawa terms of each layer exchange no energy with psi_i:
    sum psi_i G_i = 0."""
    b = O.TwoLayer(16, 16, A=0.0, sigma=0.0, amp=0.0, levels=0)
    rng = np.random.default_rng(23)
    Q1 = O.embed(rng.normal(size=(15, 15)))
    Q2 = O.embed(rng.normal(size=(15, 15)))
    psi1, psi2 = O.two_layer_cgp_psi(Q1, Q2, b)
    G1, G2 = O.two_layer_rhs(Q1, Q2, b)
    s1 = np.sum(np.abs(O.interior(psi1) * G1))
    s2 = np.sum(np.abs(O.interior(psi2) * G2))
    assert abs(np.sum(O.interior(psi1) * G1)) < 1e-12 * s1
    assert abs(np.sum(O.interior(psi2) * G2)) < 1e-12 * s2


def test_two_layer_relative_vorticity_recovered():
    """At l = 0, w_i computed from Eq. pv-non equals lap_h psi_i."""
    b = O.TwoLayer(16, 16, levels=0)
    rng = np.random.default_rng(24)
    Q1 = O.embed(rng.normal(size=(15, 15)))
    Q2 = O.embed(rng.normal(size=(15, 15)))
    psi1, psi2 = O.two_layer_cgp_psi(Q1, Q2, b)
    w1 = (O.interior(Q1) - b.Fr / b.delta * O.interior(psi2 - psi1)) / b.Ro
    assert np.allclose(w1, O.laplacian5(psi1, b.dx, b.dy), rtol=1e-10, atol=1e-9 * np.abs(w1).max())
