"""Pins of the oracle's mapping operators (Section 3.1, Eqs. res and pro).

Full weighting is exact on bilinear functions and has second moment 1/2 per
direction; bilinear prolongation reproduces bilinear functions; and the two
are adjoint up to the factor 1/4 per level (<R f, c> = 1/4 <f, P c>), so a
wrong weight in either one breaks at least one pin.
"""
import numpy as np
import pytest

from oracle import qg_oracle as O
from tests.oracle_helpers import node_coords


@pytest.mark.parametrize("nx,ny", [(8, 16), (16, 16), (32, 8)])
def test_restriction_exact_on_bilinear(nx, ny):
    X, Y = node_coords(nx, ny, 0.0, 1.0, -1.0, 1.0)
    f = 0.3 + 1.7 * X - 2.1 * Y + 0.9 * X * Y
    c = O.restrict(f)
    Xc, Yc = X[::2, ::2], Y[::2, ::2]
    assert np.allclose(c, 0.3 + 1.7 * Xc - 2.1 * Yc + 0.9 * Xc * Yc, rtol=0, atol=1e-14)


def test_restriction_second_moment():
    """R(x^2) = x^2 + h^2/2 at interior coarse nodes: sum_d w(d) d^2 = 1/2
    for the 1-D weights (1/4, 1/2, 1/4)."""
    nx, ny = 16, 16
    X, Y = node_coords(nx, ny, 0.0, 1.0, 0.0, 1.0)
    h = 1.0 / nx
    c = O.restrict(X ** 2)
    Xc = X[::2, ::2]
    assert np.allclose(c[1:-1, 1:-1], (Xc ** 2 + h ** 2 / 2)[1:-1, 1:-1], rtol=0, atol=1e-15)
    c = O.restrict(X ** 2 * Y ** 2)
    Yc = Y[::2, ::2]
    want = (Xc ** 2 + h ** 2 / 2) * (Yc ** 2 + h ** 2 / 2)
    assert np.allclose(c[1:-1, 1:-1], want[1:-1, 1:-1], rtol=0, atol=1e-15)


@pytest.mark.parametrize("mx,my", [(4, 8), (8, 8), (16, 4)])
def test_prolongation_exact_on_bilinear(mx, my):
    Xc, Yc = node_coords(mx, my, 0.0, 1.0, -0.5, 0.5)
    g = lambda X, Y: -0.4 + 2.5 * X + 0.7 * Y - 1.3 * X * Y  # noqa: E731
    f = O.prolong(g(Xc, Yc))
    X, Y = node_coords(2 * mx, 2 * my, 0.0, 1.0, -0.5, 0.5)
    assert np.allclose(f, g(X, Y), rtol=0, atol=1e-14)


def test_prolongation_values_by_hand():
    """A single unit coarse value spreads as 1, 1/2, 1/4 (Eq. pro)."""
    c = np.zeros((3, 3))
    c[1, 1] = 1.0
    f = O.prolong(c)
    want = np.zeros((5, 5))
    want[1:4, 1:4] = [[0.25, 0.5, 0.25], [0.5, 1.0, 0.5], [0.25, 0.5, 0.25]]
    assert np.array_equal(f, want)


def test_restriction_values_by_hand():
    """A single unit fine value at (2, 2) gives 4/16 at coarse (1, 1); at
    (1, 2) it gives 2/16 to coarse (1, 1) (Eq. res)."""
    f = np.zeros((9, 9))
    f[2, 2] = 1.0
    assert O.restrict(f)[1, 1] == 4.0 / 16.0
    f = np.zeros((9, 9))
    f[1, 2] = 1.0
    c = O.restrict(f)
    assert c[1, 1] == 2.0 / 16.0 and np.count_nonzero(c) == 1
    f = np.zeros((9, 9))
    f[3, 3] = 1.0
    c = O.restrict(f)
    assert c[1, 1] == c[2, 2] == c[1, 2] == c[2, 1] == 1.0 / 16.0


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_restriction_is_quarter_prolongation_transpose(levels):
    """<R^l f, c> = 4^-l <f, P^l c> for zero-wall f and c."""
    nx, ny = 32, 64
    rng = np.random.default_rng(11)
    f = O.embed(rng.normal(size=(ny - 1, nx - 1)))
    mx, my = nx >> levels, ny >> levels
    c = O.embed(rng.normal(size=(my - 1, mx - 1)))
    lhs = np.sum(O.interior(O.restrict_levels(f, levels)) * O.interior(c))
    rhs = np.sum(O.interior(f) * O.interior(O.prolong_levels(c, levels))) / 4.0 ** levels
    assert abs(lhs - rhs) <= 1e-13 * np.sum(np.abs(O.interior(f)))


def test_restriction_of_interior_never_reads_walls():
    """Interior coarse nodes depend on interior fine nodes only (the 3x3
    support of coarse node I is fine nodes 2I-1..2I+1)."""
    nx, ny = 16, 32
    f = np.zeros((ny + 1, nx + 1))
    f[0, :] = f[-1, :] = f[:, 0] = f[:, -1] = 123.0
    c = O.restrict_levels(f, 2)
    assert np.all(c[1:-1, 1:-1] == 0.0)


def smooth_vorticity(b):
    """Two low modes of the basin, zero on the walls."""
    X, Y = np.meshgrid(O.grid_x(b), O.grid_y(b))
    s = (Y - b.y0) / (b.y1 - b.y0)
    w = np.sin(np.pi * X) * np.sin(np.pi * s) + 0.5 * np.sin(2 * np.pi * X) * np.sin(3 * np.pi * s)
    w[0, :] = w[-1, :] = 0.0
    w[:, 0] = w[:, -1] = 0.0
    return w


def cgp_error_ratios(psi_fn, nx=128, ny=256, levels=(1, 2, 3)):
    """Relative distance of the projected psi (restrict, solve on the
    elliptic grid, prolong: Section 3) from the full-grid psi, per level,
    and the ratios between successive levels."""
    b0 = O.Basin(nx, ny, levels=0)
    w = smooth_vorticity(b0)
    p0 = O.cgp_psi(w, b0)
    e = [np.linalg.norm(psi_fn(w, O.with_levels(b0, l)) - p0) / np.linalg.norm(p0)
         for l in levels]
    return e, [e[k + 1] / e[k] for k in range(len(e) - 1)]


def test_cgp_projection_is_second_order_in_the_elliptic_spacing():
    """Full weighting, the 5-point solve and bilinear prolongation are each
    second order, so for a smooth field the CGP streamfunction approaches
    the full-grid one by a factor 4 per halving of the elliptic spacing."""
    e, r = cgp_error_ratios(O.cgp_psi)
    assert e[0] < 1e-3
    for q in r:
        assert 3.5 < q < 5.0, r
