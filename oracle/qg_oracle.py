"""Plain FP64 CPU oracle for the coarse grid projection (CGP) time step of
San & Staples, "An Efficient Coarse Grid Projection Method for Quasigeostrophic
Models of Large-Scale Ocean Circulation" (arXiv 1308.3290).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports, links or executes
this module; only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may.  It shares no code, table or helper with the CUDA
path.  It is written to be checked by eye against the paper, not to be fast:
every step is the definition or the algorithm step the paper states, in the
paper's order, in float64, with numpy matrix products as the only library
primitive.

Conventions (the paper's, Section 4.3): a basin has ``nx`` x ``ny`` grid
*intervals*; nodes are i = 0..nx (x) and j = 0..ny (y); the walls are the
first and last node of each direction and the unknowns are the interior nodes
i = 1..nx-1, j = 1..ny-1.  A "node array" has shape (ny+1, nx+1) and is
indexed [j, i]; an "interior array" has shape (ny-1, nx-1).

Readings of points the paper leaves open:
  * The one-layer state is the relative vorticity w = (q - y)/Ro rather than
    q itself (the two are equal in exact arithmetic, see ``rhs_q_form``).
  * Dissipation is (1/Re) times the 5-point Laplacian of the fine-grid w,
    with w = 0 on the walls (Section 2.1 boundary conditions).
  * The beta term is the Arakawa Jacobian J(psi, y) itself.
  * Kinetic energy uses one-sided differences on the grid edges.
"""
from __future__ import annotations

import functools
from dataclasses import dataclass, field, replace

import numpy as np

__all__ = [
    "Basin", "TwoLayer", "grid_y", "grid_x",
    "sine_matrix", "sine_analysis", "sine_synthesis",
    "laplacian_eigenvalues", "alpha", "poisson_solve", "elliptic_one_layer",
    "elliptic_two_layer", "restrict", "prolong", "restrict_levels",
    "prolong_levels", "arakawa", "arakawa_terms", "laplacian5",
    "forcing_one_layer", "rhs_omega", "cgp_psi", "cgp_rhs", "tvdrk3",
    "cgprk3_step", "run", "rhs_q_form", "cgprk3_step_q_form",
    "kinetic_energy", "enstrophy", "max_velocity", "cfl_dt", "adaptive_dt",
    "cgprk3_step_adaptive", "run_adaptive", "mean_psi", "mean_psi_two_layer",
    "mean_q", "mean_q_two_layer",
    "two_layer_cgp_psi", "two_layer_rhs", "cgprk3_step_two_layer",
    "interior", "embed",
]


# ---------------------------------------------------------------------------
# Problem description
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Basin:
    """One-layer barotropic basin (Section 2.1) and its CGP set-up (Section 3).

    nx, ny   : fine-grid intervals (powers of two).
    Re, Ro   : Reynolds and Rossby numbers (Eqs. Rhines, Munk).
    levels   : CGP coarsening level l; the elliptic grid is nx/2^l x ny/2^l
               (Section 3, M = 2^-l N).
    dt       : fixed time step of the TVDRK3 integrator (Section 4.2).
    amp      : amplitude multiplying the double-gyre forcing sin(pi y).
    forcing  : optional interior array that replaces amp*sin(pi y)/Ro.
    """
    nx: int
    ny: int
    Re: float = 200.0
    Ro: float = 0.0016
    levels: int = 1
    dt: float = 1e-4
    amp: float = 1.0
    x0: float = 0.0
    x1: float = 1.0
    y0: float = -1.0
    y1: float = 1.0
    forcing: np.ndarray | None = field(default=None, compare=False, repr=False)

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self) -> float:
        return (self.y1 - self.y0) / self.ny

    def coarse(self, levels: int | None = None) -> tuple[int, int, float, float]:
        """Intervals and spacings of the elliptic grid after ``levels`` halvings."""
        lv = self.levels if levels is None else levels
        f = 2 ** lv
        return self.nx // f, self.ny // f, self.dx * f, self.dy * f


@dataclass(frozen=True)
class TwoLayer:
    """Two-layer stratified basin (Section 2.2, dimensionless Eqs. ge-non and
    pv-non).  ``A`` is the lateral eddy viscosity, ``sigma`` the bottom drag,
    ``delta`` = H1/H the layer-thickness ratio."""
    nx: int
    ny: int
    Ro: float = 2.49e-4
    Fr: float = 0.087
    A: float = 3.57e-7
    sigma: float = 1.43e-3
    delta: float = 0.2
    levels: int = 1
    dt: float = 1e-5
    amp: float = 1.0
    x0: float = 0.0
    x1: float = 1.0
    y0: float = -0.5
    y1: float = 0.5

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self) -> float:
        return (self.y1 - self.y0) / self.ny

    def coarse(self, levels: int | None = None) -> tuple[int, int, float, float]:
        lv = self.levels if levels is None else levels
        f = 2 ** lv
        return self.nx // f, self.ny // f, self.dx * f, self.dy * f


def grid_x(b) -> np.ndarray:
    """Node x coordinates x_i = x0 + i dx, i = 0..nx."""
    return b.x0 + b.dx * np.arange(b.nx + 1)


def grid_y(b) -> np.ndarray:
    """Node y coordinates y_j = y0 + j dy, j = 0..ny."""
    return b.y0 + b.dy * np.arange(b.ny + 1)


def interior(a: np.ndarray) -> np.ndarray:
    """Interior part of a node array."""
    return a[1:-1, 1:-1]


def embed(a_int: np.ndarray, wall: float | np.ndarray = 0.0) -> np.ndarray:
    """Node array whose interior is ``a_int`` and whose walls hold ``wall``."""
    ny1, nx1 = a_int.shape
    out = np.empty((ny1 + 2, nx1 + 2))
    out[...] = wall
    out[1:-1, 1:-1] = a_int
    return out


# ---------------------------------------------------------------------------
# Elliptic sub-problem: fast sine transform solver (Section 4.3)
# ---------------------------------------------------------------------------

@functools.lru_cache(maxsize=16)
def _sine_matrix_cached(n: int) -> np.ndarray:
    k = np.arange(1, n, dtype=np.float64)
    s = np.sin(np.pi * np.outer(k, k) / n)
    s.setflags(write=False)
    return s


def sine_matrix(n: int) -> np.ndarray:
    """S[k-1, i-1] = sin(pi k i / n) for k, i = 1..n-1: the kernel of the sine
    sums in Eqs. ifft-1/2 and ffft-1/2 (Section 4.3)."""
    return _sine_matrix_cached(int(n))


def sine_analysis(Q: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """Eq. ifft-1: Qhat[l, k] = (2/nx)(2/ny) sum_i sum_j Q[j, i]
    sin(pi k i/nx) sin(pi l j/ny), written as the matrix product
    (2/nx)(2/ny) S_y Q S_x over interior arrays."""
    return (2.0 / nx) * (2.0 / ny) * (sine_matrix(ny) @ Q @ sine_matrix(nx))


def sine_synthesis(P: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """Eq. ffft-1: psi[j, i] = sum_k sum_l Phat[l, k] sin(pi k i/nx) sin(pi l j/ny)."""
    return sine_matrix(ny) @ P @ sine_matrix(nx)


def laplacian_eigenvalues(nx: int, ny: int, dx: float, dy: float) -> np.ndarray:
    """lambda[l-1, k-1] = (2cos(pi k/nx) - 2)/dx^2 + (2cos(pi l/ny) - 2)/dy^2,
    i.e. Eq. ialpha without its Ro factor: alpha = Ro * lambda."""
    k = np.arange(1, nx, dtype=np.float64)
    l = np.arange(1, ny, dtype=np.float64)
    lx = (2.0 * np.cos(np.pi * k / nx) - 2.0) / dx ** 2
    ly = (2.0 * np.cos(np.pi * l / ny) - 2.0) / dy ** 2
    return ly[:, None] + lx[None, :]


def alpha(nx: int, ny: int, dx: float, dy: float, Ro: float) -> np.ndarray:
    """Eq. ialpha: alpha_kl = Ro/dx^2 (2cos(pi k/nx)-2) + Ro/dy^2 (2cos(pi l/ny)-2)."""
    k = np.arange(1, nx, dtype=np.float64)
    l = np.arange(1, ny, dtype=np.float64)
    ax = Ro / dx ** 2 * (2.0 * np.cos(np.pi * k / nx) - 2.0)
    ay = Ro / dy ** 2 * (2.0 * np.cos(np.pi * l / ny) - 2.0)
    return ay[:, None] + ax[None, :]


def elliptic_one_layer(Q: np.ndarray, nx: int, ny: int, dx: float, dy: float,
                       Ro: float) -> np.ndarray:
    """Solve Ro lap(psi) = Q with psi = 0 on the walls (the one-layer form of
    Eq. sub-pr): analysis (Eq. ifft-1), psihat = Qhat/alpha (Eq. ialpha),
    synthesis (Eq. ffft-1).  Q and the result are interior arrays."""
    Qh = sine_analysis(Q, nx, ny)
    Ph = Qh / alpha(nx, ny, dx, dy, Ro)
    return sine_synthesis(Ph, nx, ny)


def poisson_solve(rhs: np.ndarray, nx: int, ny: int, dx: float, dy: float) -> np.ndarray:
    """Solve the 5-point discrete lap(psi) = rhs, psi = 0 on the walls
    (elliptic_one_layer with Ro = 1)."""
    return elliptic_one_layer(rhs, nx, ny, dx, dy, 1.0)


def elliptic_two_layer(Q1: np.ndarray, Q2: np.ndarray, nx: int, ny: int,
                       dx: float, dy: float, Ro: float, Fr: float,
                       delta: float) -> tuple[np.ndarray, np.ndarray]:
    """Coupled elliptic sub-problem of the two-layer model (Eq. sub-pr):
    analysis of both layers (Eqs. ifft-1/2), the per-mode 2x2 solution
    (Eqs. isub-1/2) with alpha from Eq. ialpha, synthesis (Eqs. ffft-1/2)."""
    Q1h = sine_analysis(Q1, nx, ny)
    Q2h = sine_analysis(Q2, nx, ny)
    a = alpha(nx, ny, dx, dy, Ro)
    f1 = Fr / delta
    f2 = Fr / (1.0 - delta)
    den = a * (a - f1 - f2)
    P1h = (a * Q1h - f2 * Q1h - f1 * Q2h) / den
    P2h = (a * Q2h - f2 * Q1h - f1 * Q2h) / den
    return sine_synthesis(P1h, nx, ny), sine_synthesis(P2h, nx, ny)


# ---------------------------------------------------------------------------
# Mapping operators (Section 3.1)
# ---------------------------------------------------------------------------

def restrict(f: np.ndarray) -> np.ndarray:
    """Full-weighting restriction, Eq. res, one level, on node arrays.

    Coarse node (I, J) sits on fine node (2I, 2J).  Interior coarse nodes take
    the 9-point weighted mean of Eq. res; the coarse wall nodes take the fine
    wall value at the same place."""
    ny, nx = f.shape[0] - 1, f.shape[1] - 1
    my, mx = ny // 2, nx // 2
    c = np.zeros((my + 1, mx + 1))
    c[0, :] = f[0, ::2]
    c[-1, :] = f[-1, ::2]
    c[:, 0] = f[::2, 0]
    c[:, -1] = f[::2, -1]

    def F(dj, di):
        # f[2J+dj, 2I+di] for every interior coarse node (J, I)
        return f[2 + dj:2 * my - 1 + dj:2, 2 + di:2 * mx - 1 + di:2]

    c[1:-1, 1:-1] = (4.0 * F(0, 0)
                     + 2.0 * (F(-1, 0) + F(1, 0) + F(0, -1) + F(0, 1))
                     + F(1, 1) + F(-1, 1) + F(1, -1) + F(-1, -1)) / 16.0
    return c


def prolong(c: np.ndarray) -> np.ndarray:
    """Bilinear prolongation, Eq. pro, one level, on node arrays: injection at
    coincident nodes, two-point means on edges, four-point means at cell
    centres."""
    my, mx = c.shape[0] - 1, c.shape[1] - 1
    f = np.zeros((2 * my + 1, 2 * mx + 1))
    f[0::2, 0::2] = c                                              # (2i, 2j)
    f[0::2, 1::2] = 0.5 * (c[:, :-1] + c[:, 1:])                   # (2i+1, 2j)
    f[1::2, 0::2] = 0.5 * (c[:-1, :] + c[1:, :])                   # (2i, 2j+1)
    f[1::2, 1::2] = 0.25 * (c[:-1, :-1] + c[:-1, 1:] + c[1:, :-1] + c[1:, 1:])
    return f


def restrict_levels(f: np.ndarray, levels: int) -> np.ndarray:
    """Eq. res applied ``levels`` times (Section 3.1, multiple coarsening)."""
    for _ in range(levels):
        f = restrict(f)
    return f


def prolong_levels(c: np.ndarray, levels: int) -> np.ndarray:
    """Eq. pro applied ``levels`` times."""
    for _ in range(levels):
        c = prolong(c)
    return c


# ---------------------------------------------------------------------------
# Spatial operators (Sections 2.1 and 4.1)
# ---------------------------------------------------------------------------

def _sh(a: np.ndarray, di: int, dj: int) -> np.ndarray:
    """a[j+dj, i+di] over the interior nodes of a node array."""
    ny, nx = a.shape[0] - 1, a.shape[1] - 1
    return a[1 + dj:ny + dj, 1 + di:nx + di]


def arakawa_terms(psi: np.ndarray, q: np.ndarray, dx: float, dy: float):
    """The three discrete Jacobians J1, J2, J3 of Eqs. j1, j2, j3 at the
    interior nodes; psi and q are node arrays, index offsets are (i, j)."""
    c = 1.0 / (4.0 * dx * dy)
    p = lambda di, dj: _sh(psi, di, dj)   # noqa: E731
    w = lambda di, dj: _sh(q, di, dj)     # noqa: E731
    J1 = c * (-(w(1, 0) - w(-1, 0)) * (p(0, 1) - p(0, -1))
              + (w(0, 1) - w(0, -1)) * (p(1, 0) - p(-1, 0)))
    J2 = c * (-w(1, 0) * (p(1, 1) - p(1, -1))
              + w(-1, 0) * (p(-1, 1) - p(-1, -1))
              + w(0, 1) * (p(1, 1) - p(-1, 1))
              - w(0, -1) * (p(1, -1) - p(-1, -1)))
    J3 = c * (-w(1, 1) * (p(0, 1) - p(1, 0))
              + w(-1, -1) * (p(-1, 0) - p(0, -1))
              + w(-1, 1) * (p(0, 1) - p(-1, 0))
              - w(1, -1) * (p(1, 0) - p(0, -1)))
    return J1, J2, J3


def arakawa(psi: np.ndarray, q: np.ndarray, dx: float, dy: float) -> np.ndarray:
    """Eq. ja1: J(psi, q) = (J1 + J2 + J3)/3 at the interior nodes."""
    J1, J2, J3 = arakawa_terms(psi, q, dx, dy)
    return (J1 + J2 + J3) / 3.0


def laplacian5(f: np.ndarray, dx: float, dy: float) -> np.ndarray:
    """Second-order 5-point Laplacian (the discrete form of Eq. ke / Eq. dis)
    at the interior nodes of a node array."""
    return ((_sh(f, 1, 0) - 2.0 * _sh(f, 0, 0) + _sh(f, -1, 0)) / dx ** 2
            + (_sh(f, 0, 1) - 2.0 * _sh(f, 0, 0) + _sh(f, 0, -1)) / dy ** 2)


def forcing_one_layer(b: Basin) -> np.ndarray:
    """Wind forcing of the w-equation on the interior nodes: the sin(pi y)
    term of the dimensionless Eq. ge divided by Ro, times ``amp``; or the
    user field ``b.forcing``."""
    if b.forcing is not None:
        return np.asarray(b.forcing, dtype=np.float64)
    y = grid_y(b)[1:-1]
    row = b.amp * np.sin(np.pi * y) / b.Ro
    return np.repeat(row[:, None], b.nx - 1, axis=1)


def rhs_omega(omega: np.ndarray, psi: np.ndarray, b: Basin,
              F: np.ndarray | None = None) -> np.ndarray:
    """G of Eq. jac for the state w = (q - y)/Ro.

    Dimensionless Eq. ge with q = Ro w + y (Eq. pv) and (delta_M/L)^3 = Ro/Re
    (Eqs. Rhines, Munk), divided by Ro:
        G = -J(psi, w) - (1/Ro) J(psi, y) + (1/Re) lap(w) + F,
    J the Arakawa Jacobian (Eq. ja1), lap the 5-point Laplacian.  omega and
    psi are node arrays with zero walls; returns the interior array."""
    dx, dy = b.dx, b.dy
    Y = np.repeat(grid_y(b)[:, None], b.nx + 1, axis=1)
    if F is None:
        F = forcing_one_layer(b)
    return (-arakawa(psi, omega, dx, dy)
            - arakawa(psi, Y, dx, dy) / b.Ro
            + laplacian5(omega, dx, dy) / b.Re
            + F)


def cgp_psi(omega: np.ndarray, b: Basin) -> np.ndarray:
    """Steps (ii)-(iv) of the CGP procedure (Section 3): restrict w to the
    elliptic grid l times (Eq. res), solve lap(psibar) = wbar there (the
    one-layer elliptic sub-problem, Section 4.3), prolong psibar l times
    (Eq. pro).  Node arrays in and out."""
    mx, my, dxc, dyc = b.coarse()
    wb = restrict_levels(omega, b.levels)
    pb = embed(poisson_solve(interior(wb), mx, my, dxc, dyc))
    return prolong_levels(pb, b.levels)


def cgp_rhs(omega: np.ndarray, b: Basin) -> np.ndarray:
    """G(w) of one CGPRK3 stage: psi from the projection, then Eq. jac."""
    return rhs_omega(omega, cgp_psi(omega, b), b)


def tvdrk3(u: np.ndarray, rhs, dt: float) -> np.ndarray:
    """Third-order TVD Runge-Kutta step (Eq. TVDRK, Section 4.2) of
    du/dt = rhs(u) on interior arrays embedded in node arrays with zero walls:
        u1 = u + dt R(u)
        u2 = 3/4 u + 1/4 u1 + 1/4 dt R(u1)
        u' = 1/3 u + 2/3 u2 + 2/3 dt R(u2)."""
    u1 = u.copy()
    u1[1:-1, 1:-1] = interior(u) + dt * rhs(u)
    u2 = u.copy()
    u2[1:-1, 1:-1] = (0.75 * interior(u) + 0.25 * interior(u1)
                      + 0.25 * dt * rhs(u1))
    u3 = u.copy()
    u3[1:-1, 1:-1] = (interior(u) / 3.0 + 2.0 / 3.0 * interior(u2)
                      + 2.0 / 3.0 * dt * rhs(u2))
    return u3


def cgprk3_step(omega: np.ndarray, b: Basin) -> np.ndarray:
    """One CGPRK3 step (Section 3.2): TVDRK3 whose every stage evaluates G
    through restriction, coarse solve and prolongation.  Node array in/out."""
    return tvdrk3(omega, lambda w: cgp_rhs(w, b), b.dt)


def run(omega0_int: np.ndarray, b: Basin, nsteps: int) -> np.ndarray:
    """``nsteps`` CGPRK3 steps from the interior array ``omega0_int``."""
    w = embed(np.asarray(omega0_int, dtype=np.float64))
    for _ in range(nsteps):
        w = cgprk3_step(w, b)
    return interior(w)


# ---------------------------------------------------------------------------
# The literal potential-vorticity form (Section 3.2 as printed)
# ---------------------------------------------------------------------------

def rhs_q_form(q: np.ndarray, b: Basin) -> np.ndarray:
    """G of Eq. jac for the state q itself (dimensionless Eqs. ge and pv):
    restrict q, solve lap(psibar) = (qbar - y)/Ro (the elliptic line of the
    CGPRK3 algorithm, (delta_I/L)^-2 = 1/Ro), prolong, then
        G = -J(psi, q) + (Ro/Re) lap(w) + amp sin(pi y),  w = (q - y)/Ro."""
    mx, my, dxc, dyc = b.coarse()
    qb = restrict_levels(q, b.levels)
    yc = b.y0 + dyc * np.arange(my + 1)
    rhs_c = (interior(qb) - yc[1:-1, None]) / b.Ro
    pb = embed(poisson_solve(rhs_c, mx, my, dxc, dyc))
    psi = prolong_levels(pb, b.levels)
    Y = np.repeat(grid_y(b)[:, None], b.nx + 1, axis=1)
    w = (q - Y) / b.Ro
    F = b.Ro * forcing_one_layer(b)
    return (-arakawa(psi, q, b.dx, b.dy) + b.Ro / b.Re * laplacian5(w, b.dx, b.dy) + F)


def cgprk3_step_q_form(q: np.ndarray, b: Basin) -> np.ndarray:
    """CGPRK3 step on q (node array whose walls hold q = y)."""
    return tvdrk3(q, lambda s: rhs_q_form(s, b), b.dt)


# ---------------------------------------------------------------------------
# Diagnostics (Section 5.2 kinetic energy; Section 4.2 CFL time step)
# ---------------------------------------------------------------------------

def kinetic_energy(psi: np.ndarray, dx: float, dy: float) -> float:
    """Basin-integrated kinetic energy E = 1/2 iint (psi_x^2 + psi_y^2) dx dy
    (Section 5.2), with one-sided differences on every grid edge and the
    midpoint rule: E = 1/2 dx dy [sum ((psi_{i+1,j}-psi_{i,j})/dx)^2
    + sum ((psi_{i,j+1}-psi_{i,j})/dy)^2].  psi is a node array."""
    ex = (psi[:, 1:] - psi[:, :-1]) / dx
    ey = (psi[1:, :] - psi[:-1, :]) / dy
    return 0.5 * dx * dy * (float(np.sum(ex * ex)) + float(np.sum(ey * ey)))


def enstrophy(omega: np.ndarray, dx: float, dy: float) -> float:
    """Z = 1/2 iint w^2 dx dy with the midpoint rule over the nodes."""
    return 0.5 * dx * dy * float(np.sum(omega * omega))


def max_velocity(psi: np.ndarray, dx: float, dy: float) -> float:
    """max over interior nodes of |psi_x| and |psi_y| (central differences),
    the denominator of Eq. dt."""
    px = (_sh(psi, 1, 0) - _sh(psi, -1, 0)) / (2.0 * dx)
    py = (_sh(psi, 0, 1) - _sh(psi, 0, -1)) / (2.0 * dy)
    return float(max(np.max(np.abs(px)), np.max(np.abs(py))))


def cfl_dt(psi: np.ndarray, dx: float, dy: float, c: float) -> float:
    """Eq. dt: dt = c min(dx, dy) / max(|psi_x|, |psi_y|)."""
    return c * min(dx, dy) / max_velocity(psi, dx, dy)


def adaptive_dt(psi: np.ndarray, b: Basin, c: float) -> float:
    """The step size of Eq. dt for the current streamfunction, capped by the
    basin's dt (the flow may start from rest, where Eq. dt has no bound):
    dt = min(b.dt, c min(dx, dy) / max(|psi_x|, |psi_y|))."""
    u = max_velocity(psi, b.dx, b.dy)
    return b.dt if u <= 0.0 else min(b.dt, c * min(b.dx, b.dy) / u)


def cgprk3_step_adaptive(omega: np.ndarray, b: Basin, c: float):
    """One CGPRK3 step whose dt follows Eq. dt from psi^n, the streamfunction
    of the step's first stage (CGP steps (ii)-(iv) applied to w^n).
    Returns (w^(n+1), dt)."""
    dt = adaptive_dt(cgp_psi(omega, b), b, c)
    return tvdrk3(omega, lambda w: cgp_rhs(w, b), dt), dt


def run_adaptive(omega0_int: np.ndarray, b: Basin, nsteps: int, c: float):
    """``nsteps`` adaptive CGPRK3 steps; returns (interior w, list of dt)."""
    w = embed(np.asarray(omega0_int, dtype=np.float64))
    dts = []
    for _ in range(nsteps):
        w, dt = cgprk3_step_adaptive(w, b, c)
        dts.append(dt)
    return interior(w), dts


# ---------------------------------------------------------------------------
# Two-layer model (Section 2.2, Eqs. ge-non and pv-non)
# ---------------------------------------------------------------------------

def two_layer_cgp_psi(Q1: np.ndarray, Q2: np.ndarray, b: TwoLayer):
    """Restrict Q_i = q_i - y (Eq. res), solve the coupled sub-problem on the
    elliptic grid (Eqs. sub-pr, isub-1/2), prolong both psi_i (Eq. pro)."""
    mx, my, dxc, dyc = b.coarse()
    q1b = restrict_levels(Q1, b.levels)
    q2b = restrict_levels(Q2, b.levels)
    p1, p2 = elliptic_two_layer(interior(q1b), interior(q2b), mx, my, dxc, dyc,
                                b.Ro, b.Fr, b.delta)
    return prolong_levels(embed(p1), b.levels), prolong_levels(embed(p2), b.levels)


def two_layer_rhs(Q1: np.ndarray, Q2: np.ndarray, b: TwoLayer):
    """Right-hand sides of Eq. ge-non for Q_i = q_i - y:
        G_1 = -J(psi_1, Q_1) - J(psi_1, y) + A lap(w_1) + amp sin(2 pi y)
        G_2 = -J(psi_2, Q_2) - J(psi_2, y) + A lap(w_2) - sigma w_2
    with w_i = lap(psi_i) recovered from Eq. pv-non on the fine grid,
    w_1 = [Q_1 - Fr/delta (psi_2 - psi_1)]/Ro,
    w_2 = [Q_2 - Fr/(1-delta) (psi_1 - psi_2)]/Ro, and w_i = 0 on the walls
    (free slip, Section 2.2)."""
    psi1, psi2 = two_layer_cgp_psi(Q1, Q2, b)
    dx, dy = b.dx, b.dy
    Y = np.repeat(grid_y(b)[:, None], b.nx + 1, axis=1)
    w1 = np.zeros_like(Q1)
    w2 = np.zeros_like(Q2)
    w1[1:-1, 1:-1] = (interior(Q1) - b.Fr / b.delta * interior(psi2 - psi1)) / b.Ro
    w2[1:-1, 1:-1] = (interior(Q2) - b.Fr / (1.0 - b.delta) * interior(psi1 - psi2)) / b.Ro
    y = grid_y(b)[1:-1]
    F1 = np.repeat((b.amp * np.sin(2.0 * np.pi * y))[:, None], b.nx - 1, axis=1)
    G1 = (-arakawa(psi1, Q1, dx, dy) - arakawa(psi1, Y, dx, dy)
          + b.A * laplacian5(w1, dx, dy) + F1)
    G2 = (-arakawa(psi2, Q2, dx, dy) - arakawa(psi2, Y, dx, dy)
          + b.A * laplacian5(w2, dx, dy) - b.sigma * interior(w2))
    return G1, G2


def cgprk3_step_two_layer(Q1: np.ndarray, Q2: np.ndarray, b: TwoLayer):
    """One CGPRK3 step of the two-layer model: TVDRK3 (Eq. TVDRK) applied to
    both layers with the coupled right-hand side."""
    dt = b.dt

    def upd(a1, a2, c1, c2, s):
        G1, G2 = two_layer_rhs(c1, c2, b)
        n1, n2 = a1.copy(), a2.copy()
        n1[1:-1, 1:-1] = s[0] * interior(a1) + s[1] * (interior(c1) + dt * G1)
        n2[1:-1, 1:-1] = s[0] * interior(a2) + s[1] * (interior(c2) + dt * G2)
        return n1, n2

    a1, a2 = upd(Q1, Q2, Q1, Q2, (0.0, 1.0))
    b1, b2 = upd(Q1, Q2, a1, a2, (0.75, 0.25))
    return upd(Q1, Q2, b1, b2, (1.0 / 3.0, 2.0 / 3.0))


def with_levels(b, levels: int):
    """Copy of a basin description with another coarsening level."""
    return replace(b, levels=levels)


# ---------------------------------------------------------------------------
# Time means (Section 5.1: the time-mean streamfunction of the statistically
# steady flow)
# ---------------------------------------------------------------------------

def mean_psi(omega0_int: np.ndarray, b: Basin, n0: int, n1: int) -> np.ndarray:
    """Mean of psi^n = CGP steps (ii)-(iv) applied to w^n over the steps
    n = n0..n1-1 of the run from w^0 = omega0 (interior array out)."""
    w = embed(np.asarray(omega0_int, dtype=np.float64))
    acc = np.zeros_like(w)
    for n in range(n1):
        if n >= n0:
            acc += cgp_psi(w, b)
        w = cgprk3_step(w, b)
    return interior(acc) / (n1 - n0)


def mean_psi_two_layer(Q1_int: np.ndarray, Q2_int: np.ndarray, b: TwoLayer, n0: int,
                       n1: int):
    """Two-layer version of ``mean_psi``: (mean psi_1, mean psi_2)."""
    a1 = embed(np.asarray(Q1_int, dtype=np.float64))
    a2 = embed(np.asarray(Q2_int, dtype=np.float64))
    s1 = np.zeros_like(a1)
    s2 = np.zeros_like(a2)
    for n in range(n1):
        if n >= n0:
            p1, p2 = two_layer_cgp_psi(a1, a2, b)
            s1 += p1
            s2 += p2
        a1, a2 = cgprk3_step_two_layer(a1, a2, b)
    return interior(s1) / (n1 - n0), interior(s2) / (n1 - n0)


def mean_q(omega0_int: np.ndarray, b: Basin, n0: int, n1: int) -> np.ndarray:
    """Time-mean potential vorticity of Section 5.1 over the steps
    n = n0..n1-1: the mean of q^n = Ro w^n + y (Eq. pv with
    (delta_I/L)^2 = Ro, Eq. Rhines) at the interior nodes."""
    w = embed(np.asarray(omega0_int, dtype=np.float64))
    y = grid_y(b)[1:-1]
    acc = np.zeros((b.ny - 1, b.nx - 1))
    for n in range(n1):
        if n >= n0:
            acc += b.Ro * interior(w) + y[:, None]
        w = cgprk3_step(w, b)
    return acc / (n1 - n0)


def mean_q_two_layer(Q1_int: np.ndarray, Q2_int: np.ndarray, b: TwoLayer, n0: int, n1: int):
    """Two-layer version of ``mean_q``: the means of q_i^n = Q_i^n + y
    (Section 4.3's variable Q_i = q_i - y)."""
    a1 = embed(np.asarray(Q1_int, dtype=np.float64))
    a2 = embed(np.asarray(Q2_int, dtype=np.float64))
    y = grid_y(b)[1:-1][:, None]
    s1 = np.zeros((b.ny - 1, b.nx - 1))
    s2 = np.zeros_like(s1)
    for n in range(n1):
        if n >= n0:
            s1 += interior(a1) + y
            s2 += interior(a2) + y
        a1, a2 = cgprk3_step_two_layer(a1, a2, b)
    return s1 / (n1 - n0), s2 / (n1 - n0)
