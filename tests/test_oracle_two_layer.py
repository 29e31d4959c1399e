"""Pins of the oracle's two-layer model (Section 2.2, Eqs. sub-pr, isub-1/2).

The coupled spectral solve is checked against a dense block solve of Eq.
sub-pr and against the barotropic/baroclinic modal split it is algebraically
equal to; the right-hand side against the layer-wise energy exchange that the
Arakawa scheme forbids.
"""
import dataclasses

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


# ---------------------------------------------------------------------------
# Pins of the dissipation, drag, forcing and time stepping of the two-layer
# model.  Each check takes the function under test as an argument, so that
# tests/test_oracle_mutations.py can hand it copies with planted mistakes.
# ---------------------------------------------------------------------------

def decoupled_limit_error(step2, levels, nsteps=4):
    """Relative difference between the two-layer step ``step2`` with Fr = 0
    and sigma = 0 and the one-layer oracle.

    With Fr = 0, Eq. pv-non gives Q_i = Ro lap psi_i, so each layer obeys
    Eq. ge-non on its own: dividing by Ro, w_i = Q_i/Ro follows the one-layer
    vorticity equation with Re = Ro/A (Table 2 lists Re = 697.16 = Ro/A), the
    square basin of Section 2.2, and the forcing sin(2 pi y)/Ro (times amp) on
    layer 1 and none on layer 2.  That equation is pinned term by term by the
    one-layer tests, and its time stepping by the TVDRK3 pins."""
    nx, ny = 16, 16
    b2 = O.TwoLayer(nx, ny, Fr=0.0, sigma=0.0, amp=1.3, levels=levels, dt=5e-5)
    rng = np.random.default_rng(31 + levels)
    w1 = 20.0 * rng.normal(size=(ny - 1, nx - 1))
    w2 = 20.0 * rng.normal(size=(ny - 1, nx - 1))
    Q1, Q2 = O.embed(b2.Ro * w1), O.embed(b2.Ro * w2)
    for _ in range(nsteps):
        Q1, Q2 = step2(Q1, Q2, b2)
    y = O.grid_y(b2)[1:-1]
    F1 = np.repeat((b2.amp * np.sin(2.0 * np.pi * y) / b2.Ro)[:, None], nx - 1, axis=1)
    errs = []
    for w0, F, Q in ((w1, F1, Q1), (w2, np.zeros_like(F1), Q2)):
        b1 = O.Basin(nx, ny, Re=b2.Ro / b2.A, Ro=b2.Ro, levels=levels, dt=b2.dt,
                     y0=b2.y0, y1=b2.y1, forcing=F)
        ref = O.run(w0, b1, nsteps)
        got = O.interior(Q) / b2.Ro
        errs.append(float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
    return max(errs)


def drag_rates(step2, h=1e-6):
    """Energy rates of the two layers with Fr = A = amp = 0 at l = 0, from a
    Richardson-extrapolated difference quotient of the kinetic energy of
    Section 5.2 over one step of size h and h/2.

    The Arakawa terms exchange no energy (sum psi J(psi, .) = 0), so with
    the drag -sigma lap psi_2 of Eq. ge-non the only source is
    dE_2/dt = -(1/Ro) sum psi_2 (-sigma lap psi_2) dx dy = -(2 sigma/Ro) E_2
    (E = -1/2 dx dy sum psi lap psi, summation by parts), and dE_1/dt = 0.
    Returns (rate_1/E_2, rate_2/E_2, -2 sigma/Ro)."""
    b = O.TwoLayer(16, 16, Fr=0.0, A=0.0, amp=0.0, levels=0)
    rng = np.random.default_rng(37)
    Q1 = O.embed(b.Ro * rng.normal(size=(15, 15)))
    Q2 = O.embed(b.Ro * rng.normal(size=(15, 15)))

    def energies(a1, a2):
        p1, p2 = O.two_layer_cgp_psi(a1, a2, b)
        return (O.kinetic_energy(p1, b.dx, b.dy), O.kinetic_energy(p2, b.dx, b.dy))

    E0 = energies(Q1, Q2)

    def quotient(dt):
        n1, n2 = step2(Q1, Q2, dataclasses.replace(b, dt=dt))
        E = energies(n1, n2)
        return [(E[k] - E0[k]) / dt for k in (0, 1)]

    d1, d2 = quotient(h), quotient(h / 2)
    r = [2.0 * d2[k] - d1[k] for k in (0, 1)]
    return r[0] / E0[1], r[1] / E0[1], -2.0 * b.sigma / b.Ro


# sin(2 pi y) at the interior rows y_j = -1/2 + j/8 of an 8 x 8 square basin
# (Section 2.2), j = 1..7, written out from the unit circle.
_S2 = np.sqrt(2.0) / 2.0
SIN_2PI_Y_8 = np.array([-_S2, -1.0, -_S2, 0.0, _S2, 1.0, _S2])


def term_errors(rhs2):
    """Each term of Eq. ge-non, isolated by switching the others off, against
    its definition at l = 0 (where the coupled solve makes Eq. pv-non exact,
    w_i = lap_h psi_i, Fr != 0):
      viscosity  A lap^2 psi_i = A lap_h(lap_h psi_i), w = 0 on the walls;
      drag       -sigma lap_h psi_2 on layer 2 only;
      forcing    amp sin(2 pi y) on layer 1 only, at the values above.
    Returns the largest relative error."""
    b = O.TwoLayer(8, 8, levels=0, amp=1.7)
    rng = np.random.default_rng(41)
    Q1 = O.embed(b.Ro * 30.0 * rng.normal(size=(7, 7)))
    Q2 = O.embed(b.Ro * 30.0 * rng.normal(size=(7, 7)))
    psi = O.two_layer_cgp_psi(Q1, Q2, b)
    R = dataclasses.replace
    base = rhs2(Q1, Q2, R(b, A=0.0, sigma=0.0, amp=0.0))
    lap = lambda f: O.laplacian5(f, b.dx, b.dy)   # noqa: E731
    want = {
        "A": [b.A * lap(O.embed(lap(p))) for p in psi],
        "sigma": [np.zeros((7, 7)), -b.sigma * lap(psi[1])],
        "amp": [np.repeat((b.amp * SIN_2PI_Y_8)[:, None], 7, axis=1), np.zeros((7, 7))],
    }
    worst = 0.0
    for name, terms in want.items():
        on = {"A": 0.0, "sigma": 0.0, "amp": 0.0}
        on[name] = getattr(b, name)
        G = rhs2(Q1, Q2, R(b, **on))
        scale = max(np.abs(t).max() for t in terms)
        for k in (0, 1):
            worst = max(worst, float(np.abs(G[k] - base[k] - terms[k]).max() / scale))
    return worst


@pytest.mark.parametrize("levels", [0, 1])
def test_decoupled_limit_is_the_one_layer_model(levels):
    assert decoupled_limit_error(O.cgprk3_step_two_layer, levels) <= 1e-11


def test_bottom_drag_energy_decay_rate():
    r1, r2, want = drag_rates(O.cgprk3_step_two_layer)
    assert abs(r2 - want) <= 1e-6 * abs(want)
    assert abs(r1) <= 1e-6 * abs(want)


def test_two_layer_terms_one_by_one():
    assert term_errors(O.two_layer_rhs) <= 1e-9


# sin(pi y) at the interior rows y_j = -1 + j/6 of a basin on [-1, 1] with
# 12 intervals in y (Section 2.1), j = 1..11.
_S3 = np.sqrt(3.0) / 2.0
SIN_PI_Y_12 = np.array([-0.5, -_S3, -1.0, -_S3, -0.5, 0.0, 0.5, _S3, 1.0, _S3, 0.5])


def forcing_error(forcing):
    """The one-layer wind forcing of the w-equation, a sin(pi y)/Ro (Eq. ge
    divided by Ro, Eq. forc), against the values of sin(pi y) at rows where it
    is known in closed form, on two basins; and a user field passed through
    unchanged."""
    worst = 0.0
    for nx, ny, amp, Ro, table in ((8, 12, 1.7, 0.0016, SIN_PI_Y_12),
                                   (16, 4, 0.6, 0.0025, np.array([-1.0, 0.0, 1.0]))):
        b = O.Basin(nx, ny, Ro=Ro, amp=amp)
        want = np.repeat((amp * table / Ro)[:, None], nx - 1, axis=1)
        got = forcing(b)
        if got.shape != want.shape:
            return np.inf
        worst = max(worst, float(np.abs(got - want).max() / np.abs(want).max()))
    user = np.arange(21.0).reshape(3, 7)
    got = forcing(O.Basin(8, 4, forcing=user))
    if got.shape != user.shape or not np.array_equal(got, user):
        return np.inf
    return worst


def test_one_layer_forcing_closed_form():
    assert forcing_error(O.forcing_one_layer) <= 1e-14
