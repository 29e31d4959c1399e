"""The oracle pins catch plausible mistakes.

Each case plants one mistake in a copy of an oracle function (a dropped term,
a flipped sign, a wrong weight or index, a transposed operand) on the CPU and
checks that the pin written for that function rejects it.  Nothing here
touches the CUDA path.
"""
import numpy as np

from oracle import qg_oracle as O
from tests.oracle_helpers import dense_laplacian


def _fields(nx=16, ny=32, seed=0):
    rng = np.random.default_rng(seed)
    a = O.embed(rng.normal(size=(ny - 1, nx - 1)))
    b = O.embed(rng.normal(size=(ny - 1, nx - 1)))
    return a, b


def _conserves(jac):
    psi, w = _fields()
    J = jac(psi, w, 1 / 16, 1 / 16)
    scale = np.sum(np.abs(J)) * max(np.abs(psi).max(), np.abs(w).max())
    return (abs(np.sum(O.interior(psi) * J)) < 1e-14 * scale
            and abs(np.sum(O.interior(w) * J)) < 1e-14 * scale)


def test_arakawa_pins_reject_mistakes():
    assert _conserves(O.arakawa)

    def dropped_J3(psi, q, dx, dy):
        J1, J2, _ = O.arakawa_terms(psi, q, dx, dy)
        return (J1 + J2) / 2.0

    def flipped_J2(psi, q, dx, dy):
        J1, J2, J3 = O.arakawa_terms(psi, q, dx, dy)
        return (J1 - J2 + J3) / 3.0

    assert not _conserves(dropped_J3)
    assert not _conserves(flipped_J2)
    # swapped operands conserve but change the sign: the closed form of
    # J(psi, y) catches it
    nx, ny = 16, 32
    dx, dy = 1 / 16, 2 / 32
    psi = np.random.default_rng(9).normal(size=(ny + 1, nx + 1))
    Y = np.repeat((-1.0 + dy * np.arange(ny + 1))[:, None], nx + 1, axis=1)
    c = (psi[:, 2:] - psi[:, :-2]) / (2 * dx)
    want = (4 * c[1:-1] + c[2:] + c[:-2]) / 6.0
    assert np.allclose(O.arakawa(psi, Y, dx, dy), want, atol=1e-11)
    assert not np.allclose(O.arakawa(Y, psi, dx, dy), want, atol=1e-6)


def test_solver_pins_reject_mistakes():
    nx, ny = 8, 16
    dx, dy = 1 / 8, 1 / 16
    rhs = np.random.default_rng(6).normal(size=(ny - 1, nx - 1))
    ref = np.linalg.solve(dense_laplacian(nx, ny, dx, dy), rhs.ravel()).reshape(rhs.shape)

    def good(r):
        return O.poisson_solve(r, nx, ny, dx, dy)

    def swapped_spacing(r):
        Ph = O.sine_analysis(r, nx, ny) / O.laplacian_eigenvalues(nx, ny, dy, dx)
        return O.sine_synthesis(Ph, nx, ny)

    def half_norm(r):
        Ph = 0.5 * O.sine_analysis(r, nx, ny) / O.laplacian_eigenvalues(nx, ny, dx, dy)
        return O.sine_synthesis(Ph, nx, ny)

    def ok(f):
        return np.linalg.norm(f(rhs) - ref) <= 1e-12 * np.linalg.norm(ref)

    assert ok(good)
    assert not ok(swapped_spacing)
    assert not ok(half_norm)


def test_transfer_pins_reject_mistakes():
    nx, ny, lv = 32, 64, 1
    rng = np.random.default_rng(11)
    f = O.embed(rng.normal(size=(ny - 1, nx - 1)))
    c = O.embed(rng.normal(size=(ny // 2 - 1, nx // 2 - 1)))

    def adjoint_ok(R, P):
        lhs = np.sum(O.interior(R(f)) * O.interior(c))
        rhs = np.sum(O.interior(f) * O.interior(P(c))) / 4.0
        return abs(lhs - rhs) <= 1e-13 * np.sum(np.abs(O.interior(f)))

    def corner_weight_2(fa):
        out = O.restrict(fa)
        g = np.zeros_like(fa)
        g[1:-1, 1:-1] = fa[1:-1, 1:-1]
        # add an extra 1/16 of one corner neighbour: a wrong corner weight
        out[1:-1, 1:-1] += g[3::2, 3::2][: out.shape[0] - 2, : out.shape[1] - 2] / 16.0
        return out

    def prolong_no_centre_avg(ca):
        out = O.prolong(ca)
        out[1::2, 1::2] = ca[:-1, :-1]
        return out

    assert adjoint_ok(O.restrict, O.prolong)
    assert not adjoint_ok(corner_weight_2, O.prolong)
    assert not adjoint_ok(O.restrict, prolong_no_centre_avg)


def test_time_pins_reject_mistakes():
    def amp(step, z):
        u = np.zeros((3, 3))
        u[1, 1] = 1.0
        return step(u, lambda s: (z / 0.01) * O.interior(s), 0.01)[1, 1]

    def wrong_stage2(u, rhs, dt):
        u1 = u.copy()
        u1[1:-1, 1:-1] = O.interior(u) + dt * rhs(u)
        u2 = u.copy()
        u2[1:-1, 1:-1] = 0.5 * O.interior(u) + 0.5 * O.interior(u1) + 0.25 * dt * rhs(u1)
        u3 = u.copy()
        u3[1:-1, 1:-1] = O.interior(u) / 3 + 2 / 3 * O.interior(u2) + 2 / 3 * dt * rhs(u2)
        return u3

    z = -0.3
    want = 1 + z + z * z / 2 + z ** 3 / 6
    assert abs(amp(O.tvdrk3, z) - want) < 1e-14
    assert abs(amp(wrong_stage2, z) - want) > 1e-4


def test_adjoint_pins_reject_mistakes():
    """The forward-difference pin of rhs_adjoint rejects a flipped beta term,
    a missing projection and transposed Jacobian operands."""
    from oracle import qg_adjoint as AD

    b = O.Basin(16, 32, levels=1)
    rng = np.random.default_rng(21)
    w = O.embed(20.0 * rng.normal(size=(31, 15)))
    dw = O.embed(rng.normal(size=(31, 15)))
    lam = O.embed(rng.normal(size=(31, 15)))
    eps = 1e-3
    dG = (O.cgp_rhs(w + eps * dw, b) - O.cgp_rhs(w - eps * dw, b)) / (2 * eps)
    lhs = np.sum(dG * O.interior(lam))
    psi = O.cgp_psi(w, b)

    def ok(adj):
        rhs = np.sum(O.interior(dw) * adj(lam, w, psi, b))
        return abs(lhs - rhs) <= 1e-9 * np.sqrt(np.sum(dG ** 2) * np.sum(lam ** 2))

    def flipped_beta(la, wv, ps, bb):
        t = O.arakawa(wv, la, bb.dx, bb.dy) + AD.beta_jacobian(la, bb) / bb.Ro
        return (O.arakawa(ps, la, bb.dx, bb.dy) + O.laplacian5(la, bb.dx, bb.dy) / bb.Re
                - O.interior(O.cgp_psi(O.embed(t), bb)))

    def no_projection(la, wv, ps, bb):
        t = O.arakawa(wv, la, bb.dx, bb.dy) - AD.beta_jacobian(la, bb) / bb.Ro
        return (O.arakawa(ps, la, bb.dx, bb.dy) + O.laplacian5(la, bb.dx, bb.dy) / bb.Re - t)

    def transposed_operands(la, wv, ps, bb):
        t = O.arakawa(wv, la, bb.dx, bb.dy) - AD.beta_jacobian(la, bb) / bb.Ro
        return (O.arakawa(la, ps, bb.dx, bb.dy) + O.laplacian5(la, bb.dx, bb.dy) / bb.Re
                - O.interior(O.cgp_psi(O.embed(t), bb)))

    assert ok(AD.rhs_adjoint)
    assert not ok(flipped_beta)
    assert not ok(no_projection)
    assert not ok(transposed_operands)


def test_two_layer_solve_pins_reject_mistakes():
    """The dense block solve of Eq. sub-pr rejects swapped layer-thickness
    factors and a flipped coupling sign in Eqs. isub-1/2."""
    nx, ny = 8, 16
    dx, dy = 1.0 / nx, 2.0 / ny
    Ro, Fr, d = 2.49e-4, 0.087, 0.2
    rng = np.random.default_rng(23)
    Q1 = rng.normal(size=(ny - 1, nx - 1))
    Q2 = rng.normal(size=(ny - 1, nx - 1))
    Lm = Ro * dense_laplacian(nx, ny, dx, dy)
    I = np.eye(Lm.shape[0])
    f1, f2 = Fr / d, Fr / (1 - d)
    M = np.block([[Lm - f1 * I, f1 * I], [f2 * I, Lm - f2 * I]])
    sol = np.linalg.solve(M, np.concatenate([Q1.ravel(), Q2.ravel()]))

    def ok(solve):
        p1, p2 = solve(Q1, Q2)
        got = np.concatenate([p1.ravel(), p2.ravel()])
        return np.linalg.norm(got - sol) <= 1e-12 * np.linalg.norm(sol)

    def spectral(c1, c2, sign):
        def solve(A, B):
            Ah, Bh = O.sine_analysis(A, nx, ny), O.sine_analysis(B, nx, ny)
            a = O.alpha(nx, ny, dx, dy, Ro)
            den = a * (a - c1 - c2)
            P1 = (a * Ah - c2 * Ah + sign * c1 * Bh) / den
            P2 = (a * Bh - c2 * Ah + sign * c1 * Bh) / den
            return O.sine_synthesis(P1, nx, ny), O.sine_synthesis(P2, nx, ny)
        return solve

    assert ok(lambda A, B: O.elliptic_two_layer(A, B, nx, ny, dx, dy, Ro, Fr, d))
    assert ok(spectral(f1, f2, -1.0))          # the same algebra, restated
    assert not ok(spectral(f2, f1, -1.0))      # thickness factors swapped
    assert not ok(spectral(f1, f2, +1.0))      # coupling sign flipped


def test_energy_pins_reject_mistakes():
    """The summation-by-parts identity of the kinetic energy rejects central
    differences and a dropped y-edge sum."""
    b = O.Basin(32, 64, levels=0)
    w = O.embed(np.random.default_rng(24).normal(size=(63, 31)))
    psi = O.cgp_psi(w, b)
    target = -0.5 * b.dx * b.dy * np.sum(O.interior(psi) * O.laplacian5(psi, b.dx, b.dy))

    def ok(E):
        return abs(E(psi, b.dx, b.dy) - target) <= 1e-12 * abs(target)

    def central(p, dx, dy):
        ex = (p[1:-1, 2:] - p[1:-1, :-2]) / (2 * dx)
        ey = (p[2:, 1:-1] - p[:-2, 1:-1]) / (2 * dy)
        return 0.5 * dx * dy * float(np.sum(ex * ex) + np.sum(ey * ey))

    def x_edges_only(p, dx, dy):
        ex = (p[:, 1:] - p[:, :-1]) / dx
        return 0.5 * dx * dy * float(np.sum(ex * ex))

    assert ok(O.kinetic_energy)
    assert not ok(central)
    assert not ok(x_edges_only)


def test_cfl_pins_reject_mistakes():
    """The closed form of max |grad psi| on a sine mode rejects one-sided
    differences and a dropped factor 2 in the central difference."""
    nx, ny = 32, 64
    dx, dy = 1.0 / nx, 2.0 / ny
    i = np.arange(nx + 1)[None, :]
    j = np.arange(ny + 1)[:, None]
    psi = 1.5 * np.sin(np.pi * i / nx) * np.sin(np.pi * j / ny)
    ux = 1.5 * np.cos(np.pi / nx) * np.sin(np.pi / nx) / dx
    uy = 1.5 * np.cos(np.pi / ny) * np.sin(np.pi / ny) / dy
    u = max(ux, uy)

    def ok(mv):
        return abs(mv(psi, dx, dy) - u) <= 1e-13 * u

    def one_sided(p, dx, dy):
        px = (p[1:-1, 2:] - p[1:-1, 1:-1]) / dx
        py = (p[2:, 1:-1] - p[1:-1, 1:-1]) / dy
        return float(max(np.abs(px).max(), np.abs(py).max()))

    def no_half(p, dx, dy):
        px = (p[1:-1, 2:] - p[1:-1, :-2]) / dx
        py = (p[2:, 1:-1] - p[:-2, 1:-1]) / dy
        return float(max(np.abs(px).max(), np.abs(py).max()))

    assert ok(O.max_velocity)
    assert not ok(one_sided)
    assert not ok(no_half)


def test_projection_order_pin_rejects_piecewise_constant_prolongation():
    """Prolonging psi by copying each coarse value to its fine cell (instead
    of Eq. pro's bilinear averages) drops the CGP projection to first order,
    which the order pin rejects."""
    from tests.test_oracle_transfer import cgp_error_ratios

    def copy_prolong(c):
        f = np.zeros((2 * c.shape[0] - 1, 2 * c.shape[1] - 1))
        f[::2, ::2] = c
        f[1::2, ::2] = c[:-1, :]
        f[::2, 1::2] = c[:, :-1]
        f[1::2, 1::2] = c[:-1, :-1]
        f[0, :] = f[-1, :] = 0.0
        f[:, 0] = f[:, -1] = 0.0
        return f

    def psi_copy(w, b):
        mx, my = b.nx >> b.levels, b.ny >> b.levels
        s = float(1 << b.levels)
        wb = O.restrict_levels(w, b.levels)
        p = O.embed(O.poisson_solve(O.interior(wb), mx, my, b.dx * s, b.dy * s))
        for _ in range(b.levels):
            p = copy_prolong(p)
        return p

    _, r = cgp_error_ratios(psi_copy)
    assert not all(3.5 < q < 5.0 for q in r), r


def _two_layer_rhs_variant(drag=-1.0, drag_layer=2, visc=1.0, k_forcing=2.0, swap_fr=False):
    """The right-hand side of Eq. ge-non restated with switches for planted
    mistakes; with the defaults it is the oracle's algebra."""
    def rhs(Q1, Q2, b):
        psi1, psi2 = O.two_layer_cgp_psi(Q1, Q2, b)
        Y = np.repeat(O.grid_y(b)[:, None], b.nx + 1, axis=1)
        f1, f2 = b.Fr / b.delta, b.Fr / (1.0 - b.delta)
        if swap_fr:
            f1, f2 = f2, f1
        w1 = O.embed((O.interior(Q1) - f1 * O.interior(psi2 - psi1)) / b.Ro)
        w2 = O.embed((O.interior(Q2) - f2 * O.interior(psi1 - psi2)) / b.Ro)
        y = O.grid_y(b)[1:-1]
        F1 = np.repeat((b.amp * np.sin(k_forcing * np.pi * y))[:, None], b.nx - 1, axis=1)
        A = visc * b.A
        G1 = (-O.arakawa(psi1, Q1, b.dx, b.dy) - O.arakawa(psi1, Y, b.dx, b.dy)
              + A * O.laplacian5(w1, b.dx, b.dy) + F1)
        G2 = (-O.arakawa(psi2, Q2, b.dx, b.dy) - O.arakawa(psi2, Y, b.dx, b.dy)
              + A * O.laplacian5(w2, b.dx, b.dy))
        if drag_layer == 2:
            G2 = G2 + drag * b.sigma * O.interior(w2)
        else:
            G1 = G1 + drag * b.sigma * O.interior(w1)
        return G1, G2
    return rhs


def _two_layer_step_variant(rhs, weights=((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))):
    """TVDRK3 (Eq. TVDRK) over both layers with a pluggable right-hand side
    and stage weights."""
    def step(Q1, Q2, b):
        def upd(a1, a2, c1, c2, s):
            G1, G2 = rhs(c1, c2, b)
            n1 = O.embed(s[0] * O.interior(a1) + s[1] * (O.interior(c1) + b.dt * G1))
            n2 = O.embed(s[0] * O.interior(a2) + s[1] * (O.interior(c2) + b.dt * G2))
            return n1, n2
        a1, a2 = upd(Q1, Q2, Q1, Q2, weights[0])
        b1, b2 = upd(Q1, Q2, a1, a2, weights[1])
        return upd(Q1, Q2, b1, b2, weights[2])
    return step


def test_two_layer_model_pins_reject_mistakes():
    """The decoupled limit, the drag energy-decay rate and the term-by-term
    pins of the two-layer model reject a flipped or misplaced drag, a wrong
    viscosity factor, the one-layer forcing wavenumber, swapped thickness
    factors in the recovered vorticity and a wrong TVDRK3 stage weight."""
    from tests.test_oracle_two_layer import decoupled_limit_error, drag_rates, term_errors

    def pins(rhs, weights=None):
        step = (_two_layer_step_variant(rhs) if weights is None
                else _two_layer_step_variant(rhs, weights))
        r1, r2, want = drag_rates(step)
        return {
            "decoupled": decoupled_limit_error(step, 1) <= 1e-11,
            "drag": abs(r2 - want) <= 1e-6 * abs(want) and abs(r1) <= 1e-6 * abs(want),
            "terms": term_errors(rhs) <= 1e-9,
        }

    assert all(pins(_two_layer_rhs_variant()).values())          # the same algebra, restated
    assert not pins(_two_layer_rhs_variant(drag=+1.0))["drag"]
    assert not pins(_two_layer_rhs_variant(drag_layer=1))["drag"]
    assert not pins(_two_layer_rhs_variant(drag=+1.0))["terms"]
    bad_visc = pins(_two_layer_rhs_variant(visc=2.0))
    assert not bad_visc["decoupled"] and not bad_visc["terms"]
    bad_forcing = pins(_two_layer_rhs_variant(k_forcing=1.0))
    assert not bad_forcing["decoupled"] and not bad_forcing["terms"]
    assert not pins(_two_layer_rhs_variant(swap_fr=True))["terms"]
    wrong_stage = ((0.0, 1.0), (0.5, 0.5), (1.0 / 3.0, 2.0 / 3.0))
    assert not pins(_two_layer_rhs_variant(), wrong_stage)["decoupled"]


def test_forcing_pin_rejects_mistakes():
    """The closed-form values of sin(pi y) reject a cosine profile, the
    two-layer wavenumber, a forcing multiplied instead of divided by Ro and
    a dropped amplitude."""
    from tests.test_oracle_two_layer import forcing_error

    def variant(fn=np.sin, k=1.0, by_ro=True, use_amp=True):
        def forcing(b):
            if b.forcing is not None:
                return np.asarray(b.forcing, dtype=np.float64)
            y = O.grid_y(b)[1:-1]
            a = b.amp if use_amp else 1.0
            row = a * fn(k * np.pi * y) * (1.0 / b.Ro if by_ro else b.Ro)
            return np.repeat(row[:, None], b.nx - 1, axis=1)
        return forcing

    assert forcing_error(variant()) <= 1e-14
    assert forcing_error(variant(fn=np.cos)) > 1e-3
    assert forcing_error(variant(k=2.0)) > 1e-3
    assert forcing_error(variant(by_ro=False)) > 1e-3
    assert forcing_error(variant(use_amp=False)) > 1e-3


def test_mean_q_pin_rejects_mistakes():
    """The q-form pin of the time-mean potential vorticity rejects a missing
    Ro factor, a missing planetary vorticity y and y taken at shifted rows."""
    b = O.Basin(32, 64, Re=200.0, Ro=0.0016, levels=1, dt=1e-4)
    from paper_1308_3290_gb300 import inputs
    w0 = inputs.perturbation(32, 64, seed=2) * 30.0
    n0, n1 = 2, 6
    Y = np.repeat(O.grid_y(b)[:, None], b.nx + 1, axis=1)
    q = b.Ro * O.embed(w0) + Y
    acc = np.zeros((63, 31))
    for n in range(n1):
        if n >= n0:
            acc += O.interior(q)
        q = O.cgprk3_step_q_form(q, b)
    want = acc / (n1 - n0)

    def variant(scale, with_y, shift):
        w = O.embed(w0)
        y = O.grid_y(b)[1 + shift:b.ny + shift]
        out = np.zeros((63, 31))
        for n in range(n1):
            if n >= n0:
                out += scale * O.interior(w) + (y[:, None] if with_y else 0.0)
            w = O.cgprk3_step(w, b)
        return out / (n1 - n0)

    def ok(m):
        return np.abs(m - want).max() <= 1e-12 * np.abs(want).max()

    assert ok(variant(b.Ro, True, 0))
    assert not ok(variant(1.0, True, 0))
    assert not ok(variant(b.Ro, False, 0))
    assert not ok(variant(b.Ro, True, 1))
