"""Pins of the oracle's time integration (Section 4.2, Eq. TVDRK) and of the
whole CGPRK3 step (Section 3.2).

The stability polynomial of the TVDRK3 step on du/dt = lambda u, third-order
convergence, the equality of the literal q-form and the w-form the library
integrates, the l = 0 reduction of CGP to the standard solver, the discrete
energy identity behind the kinetic-energy diagnostic, and third-order
self-consistency of a full CGP trajectory under dt halving.
"""
import dataclasses

import numpy as np
import pytest

from oracle import qg_oracle as O
from paper_1308_3290_gb300 import inputs


def test_tvdrk3_stability_polynomial():
    """One step of du/dt = lambda u multiplies u by 1 + z + z^2/2 + z^3/6."""
    for z in (-0.3, 0.1, -1.7, 0.9):
        lam, dt = z / 0.01, 0.01
        u = np.zeros((3, 3))
        u[1, 1] = 1.0
        out = O.tvdrk3(u, lambda s: lam * O.interior(s), dt)
        assert abs(out[1, 1] - (1 + z + z * z / 2 + z ** 3 / 6)) < 1e-14
        assert out[0, 0] == 0.0


def test_tvdrk3_third_order():
    """du/dt = -u^2, u(0) = 1, exact u = 1/(1+t)."""
    errs = []
    for n in (10, 20, 40, 80):
        dt = 1.0 / n
        u = np.zeros((3, 3))
        u[1, 1] = 1.0
        for _ in range(n):
            u = O.tvdrk3(u, lambda s: -O.interior(s) ** 2, dt)
        errs.append(abs(u[1, 1] - 0.5))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(7.0 < r < 9.0 for r in ratios), ratios


@pytest.mark.parametrize("levels", [0, 1, 2])
def test_q_form_equals_omega_form(levels):
    """Integrating q = Ro w + y with the elliptic line (qbar - y)/Ro of the
    CGPRK3 algorithm gives the same trajectory as integrating w."""
    b = O.Basin(32, 64, Re=200.0, Ro=0.0016, levels=levels, dt=1e-4)
    w0 = inputs.perturbation(32, 64, seed=1) * 30.0
    w = O.embed(w0)
    Y = np.repeat(O.grid_y(b)[:, None], b.nx + 1, axis=1)
    q = b.Ro * w + Y
    for _ in range(20):
        w = O.cgprk3_step(w, b)
        q = O.cgprk3_step_q_form(q, b)
    wq = (q - Y) / b.Ro
    assert np.linalg.norm(O.interior(wq - w)) <= 1e-11 * np.linalg.norm(O.interior(w))


def test_level_zero_is_the_standard_solver():
    """With l = 0 the projection is the identity: psi solves lap psi = w on
    the fine grid itself."""
    b = O.Basin(16, 32, levels=0)
    w = O.embed(inputs.perturbation(16, 32, seed=2))
    psi = O.cgp_psi(w, b)
    direct = O.poisson_solve(O.interior(w), 16, 32, b.dx, b.dy)
    assert np.array_equal(O.interior(psi), direct)


def test_kinetic_energy_summation_by_parts():
    """E = 1/2 dx dy sum_edges |grad psi|^2 = -1/2 dx dy sum psi lap_h psi,
    and at l = 0 lap_h psi = w, so E = -1/2 dx dy sum psi w."""
    b = O.Basin(32, 64, levels=0)
    w = O.embed(inputs.smooth_field(32, 64, seed=3, noise=0.1))
    psi = O.cgp_psi(w, b)
    E = O.kinetic_energy(psi, b.dx, b.dy)
    assert abs(E + 0.5 * b.dx * b.dy * np.sum(O.interior(psi) * O.laplacian5(psi, b.dx, b.dy))) < 1e-13 * E
    assert abs(E + 0.5 * b.dx * b.dy * np.sum(psi * w)) < 1e-12 * E


def test_cgp_trajectory_third_order_in_time():
    """A 64x128 CGP (l = 1) trajectory to t = 0.02 from a seeded state
    converges at third order as dt halves."""
    b = O.Basin(64, 128, Re=200.0, Ro=0.0016, levels=1)
    w0 = inputs.perturbation(64, 128, seed=1) * 20.0
    T = 0.02
    sols = []
    for n in (10, 20, 40):
        sols.append(O.run(w0, dataclasses.replace(b, dt=T / n), n))
    e1 = np.linalg.norm(sols[0] - sols[1])
    e2 = np.linalg.norm(sols[1] - sols[2])
    assert 6.5 < e1 / e2 < 9.5, e1 / e2


def test_cfl_dt_formula():
    b = O.Basin(16, 32, levels=0)
    psi = np.zeros((33, 17))
    x = O.grid_x(b)
    psi[:, :] = 0.0
    psi[1:-1, 1:-1] = 3.0 * x[None, 1:-1]     # psi_x = 3 in the interior away from walls
    u = O.max_velocity(psi, b.dx, b.dy)
    assert u >= 3.0
    assert O.cfl_dt(psi, b.dx, b.dy, 0.5) == pytest.approx(0.5 * b.dx / u)


def max_velocity_of_sine_mode(nx, ny, dx, dy, a):
    """Closed form of max |psi_x|, |psi_y| (central differences over the
    interior nodes) for psi = a sin(pi i/nx) sin(pi j/ny): the x difference
    is a cos(pi i/nx) sin(pi/nx)/dx sin(pi j/ny), largest at i = 1,
    j = ny/2; the y difference likewise at i = nx/2, j = 1."""
    ux = a * np.cos(np.pi / nx) * np.sin(np.pi / nx) / dx
    uy = a * np.cos(np.pi / ny) * np.sin(np.pi / ny) / dy
    return max(ux, uy)


@pytest.mark.parametrize("nx,ny,y0,y1", [(16, 32, -1.0, 1.0), (32, 16, -1.0, 1.0),
                                         (64, 64, -0.5, 0.5)])
def test_max_velocity_and_cfl_dt_closed_form(nx, ny, y0, y1):
    """Eq. dt's denominator and step on a sine mode whose central
    differences have a closed form."""
    b = O.Basin(nx, ny, levels=0, y0=y0, y1=y1)
    i = np.arange(nx + 1)[None, :]
    j = np.arange(ny + 1)[:, None]
    a = 2.5
    psi = a * np.sin(np.pi * i / nx) * np.sin(np.pi * j / ny)
    u = max_velocity_of_sine_mode(nx, ny, b.dx, b.dy, a)
    assert O.max_velocity(psi, b.dx, b.dy) == pytest.approx(u, rel=1e-13)
    assert O.cfl_dt(psi, b.dx, b.dy, 0.7) == pytest.approx(0.7 * min(b.dx, b.dy) / u, rel=1e-13)


def test_adaptive_dt_rules():
    """Eq. dt with the cap: from rest the basin's dt; a capped step is the
    fixed step; otherwise c min(dx, dy) / max|grad psi| and the step is
    TVDRK3 with that dt."""
    b = O.Basin(32, 64, levels=1, dt=1e-3)
    w0 = O.embed(np.zeros((63, 31)))
    assert O.adaptive_dt(O.cgp_psi(w0, b), b, 0.5) == b.dt
    w = O.embed(inputs.perturbation(32, 64, seed=9) * 50.0)
    psi = O.cgp_psi(w, b)
    u = O.max_velocity(psi, b.dx, b.dy)
    c_small = 0.1 * b.dt * u / min(b.dx, b.dy)           # Eq. dt below the cap
    dt = O.adaptive_dt(psi, b, c_small)
    assert dt == pytest.approx(c_small * min(b.dx, b.dy) / u, rel=1e-15)
    assert dt < b.dt
    w1, dt1 = O.cgprk3_step_adaptive(w, b, c_small)
    assert dt1 == dt
    ref = O.tvdrk3(w, lambda s: O.cgp_rhs(s, b), dt)
    assert np.array_equal(w1, ref)
    w2, dt2 = O.cgprk3_step_adaptive(w, b, 1e9)             # capped
    assert dt2 == b.dt
    assert np.array_equal(w2, O.cgprk3_step(w, b))


@pytest.mark.parametrize("levels", [0, 1, 2])
def test_mean_psi_is_the_projection_of_the_mean_state(levels):
    """psi^n is linear in w^n (P S R), so the time mean of psi^n equals the
    projection of the time-mean state, computed here from the states of an
    independent run."""
    b = O.Basin(32, 64, levels=levels, dt=1e-4)
    w0 = inputs.perturbation(32, 64, seed=12) * 50.0
    got = O.mean_psi(w0, b, 3, 9)
    w = O.embed(w0)
    states = []
    for n in range(9):
        if n >= 3:
            states.append(w)
        w = O.cgprk3_step(w, b)
    wbar = sum(states) / len(states)
    mx, my, dxc, dyc = b.coarse()
    ref = O.interior(O.prolong_levels(O.embed(O.poisson_solve(
        O.interior(O.restrict_levels(wbar, levels)), mx, my, dxc, dyc)), levels))
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_run_adaptive_threads_states_and_steps():
    """run_adaptive is the loop of Eq. dt steps: capped (c huge) it is the
    fixed-step run exactly; below the cap each step's dt is Eq. dt of that
    step's own first streamfunction and the states follow TVDRK3 with it."""
    b = O.Basin(32, 64, levels=1, dt=1e-3)
    w0 = inputs.perturbation(32, 64, seed=31) * 50.0
    w, dts = O.run_adaptive(w0, b, 4, 1e9)
    assert dts == [b.dt] * 4
    assert np.array_equal(w, O.run(w0, b, 4))
    u0 = O.max_velocity(O.cgp_psi(O.embed(w0), b), b.dx, b.dy)
    c = 0.3 * b.dt * u0 / min(b.dx, b.dy)          # Eq. dt below the cap
    w, dts = O.run_adaptive(w0, b, 4, c)
    s = O.embed(w0)
    for k in range(4):
        psi = O.cgp_psi(s, b)
        dt = min(b.dt, c * min(b.dx, b.dy) / O.max_velocity(psi, b.dx, b.dy))
        assert dts[k] == pytest.approx(dt, rel=1e-15)
        s = O.tvdrk3(s, lambda x: O.cgp_rhs(x, b), dts[k])
    assert np.array_equal(w, O.interior(s))
    assert max(dts) < b.dt


def test_two_layer_mean_psi_is_the_projection_of_the_mean_states():
    """Both layers' psi are linear in (Q1, Q2) (restriction, the coupled solve
    of Eqs. isub-1/2, prolongation), so their time means over steps n0..n1-1
    equal the projection of the mean states of an independent run."""
    b = O.TwoLayer(32, 32, levels=1, dt=1e-4)
    Q1 = inputs.smooth_field(32, 32, seed=1, amp=0.05, noise=0.01)
    Q2 = inputs.smooth_field(32, 32, seed=2, amp=0.02, noise=0.01)
    m1, m2 = O.mean_psi_two_layer(Q1, Q2, b, 2, 7)
    a1, a2 = O.embed(Q1), O.embed(Q2)
    s1, s2 = [], []
    for n in range(7):
        if n >= 2:
            s1.append(a1)
            s2.append(a2)
        a1, a2 = O.cgprk3_step_two_layer(a1, a2, b)
    p1, p2 = O.two_layer_cgp_psi(sum(s1) / 5, sum(s2) / 5, b)
    for got, ref in ((m1, O.interior(p1)), (m2, O.interior(p2))):
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("levels", [0, 1, 2])
def test_mean_q_is_the_mean_of_the_q_form_trajectory(levels):
    """The time-mean potential vorticity from the w-form trajectory equals
    the mean of the states of the literal q-form integration (Section 3.2 as
    printed: the state q itself, walls q = y), steps n0..n1-1."""
    b = O.Basin(32, 64, Re=200.0, Ro=0.0016, levels=levels, dt=1e-4)
    w0 = inputs.perturbation(32, 64, seed=2) * 30.0
    n0, n1 = 3, 12
    got = O.mean_q(w0, b, n0, n1)
    Y = np.repeat(O.grid_y(b)[:, None], b.nx + 1, axis=1)
    q = b.Ro * O.embed(w0) + Y
    acc = np.zeros_like(got)
    for n in range(n1):
        if n >= n0:
            acc += O.interior(q)
        q = O.cgprk3_step_q_form(q, b)
    want = acc / (n1 - n0)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_mean_q_at_rest_without_forcing_is_y():
    """With no forcing and w = 0 the basin stays at rest: q = y exactly
    (Eq. pv), so its time mean is the planetary vorticity y itself."""
    b = O.Basin(16, 32, levels=1, amp=0.0)
    got = O.mean_q(np.zeros((31, 15)), b, 0, 5)
    y = -1.0 + (2.0 / 32) * np.arange(1, 32)
    assert np.array_equal(got, np.repeat(y[:, None], 15, axis=1))


def test_two_layer_mean_q_is_the_mean_state_plus_y():
    """Two layers: q_i = Q_i + y (Section 4.3); with Q_i = 0, no wind and
    rest, q_i = y in both layers."""
    b = O.TwoLayer(16, 16, amp=0.0, levels=0)
    m1, m2 = O.mean_q_two_layer(np.zeros((15, 15)), np.zeros((15, 15)), b, 0, 3)
    y = -0.5 + (1.0 / 16) * np.arange(1, 16)
    assert np.array_equal(m1, np.repeat(y[:, None], 15, axis=1)) and np.array_equal(m1, m2)
