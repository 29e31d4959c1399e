"""Pins of the oracle's fast sine-transform elliptic solver (Section 4.3,
Eqs. ifft-1/2, ialpha, ffft-1/2).

Each pin comes from outside the oracle: scipy's DST-I (a library routine the
2-D sine sum reduces to), a dense direct solve of the 5-point matrix built
from the stencil, the exact discrete eigenvectors, and the O(h^2) convergence
to a continuous solution.
"""
import numpy as np
import pytest
import scipy.fft

from oracle import qg_oracle as O
from tests.oracle_helpers import dense_laplacian


@pytest.mark.parametrize("nx,ny", [(8, 16), (16, 8), (32, 64), (64, 32)])
def test_analysis_is_scipy_dst1(nx, ny):
    """scipy's DST-I of length n-1 is 2*sum x_j sin(pi (j+1)(k+1)/n); the
    paper's analysis carries (2/nx)(2/ny), so it is dstn/(nx ny)."""
    Q = np.random.default_rng(3).normal(size=(ny - 1, nx - 1))
    ref = scipy.fft.dstn(Q, type=1) / (nx * ny)
    got = O.sine_analysis(Q, nx, ny)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("nx,ny", [(8, 16), (32, 64), (128, 64)])
def test_synthesis_inverts_analysis(nx, ny):
    Q = np.random.default_rng(4).normal(size=(ny - 1, nx - 1))
    back = O.sine_synthesis(O.sine_analysis(Q, nx, ny), nx, ny)
    assert np.max(np.abs(back - Q)) < 1e-13 * np.max(np.abs(Q))


def test_synthesis_is_scipy_dst1():
    nx, ny = 16, 32
    P = np.random.default_rng(5).normal(size=(ny - 1, nx - 1))
    ref = scipy.fft.dstn(P, type=1) / 4.0
    assert np.allclose(O.sine_synthesis(P, nx, ny), ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("nx,ny,y0,y1", [(8, 16, -1.0, 1.0), (16, 16, -0.5, 0.5),
                                         (16, 32, -0.5, 0.5)])
def test_eigenvalues_are_rayleigh_quotients(nx, ny, y0, y1):
    """sin(pi k i/nx) sin(pi l j/ny) is an exact eigenvector of the dense
    5-point matrix; its eigenvalue is Eq. ialpha / Ro."""
    dx, dy = 1.0 / nx, (y1 - y0) / ny
    Lm = dense_laplacian(nx, ny, dx, dy)
    lam = O.laplacian_eigenvalues(nx, ny, dx, dy)
    i = np.arange(1, nx)
    j = np.arange(1, ny)
    for k, l in [(1, 1), (2, 5), (nx - 1, 1), (3, ny - 1), (nx - 1, ny - 1)]:
        v = (np.sin(np.pi * l * j / ny)[:, None] * np.sin(np.pi * k * i / nx)[None, :]).ravel()
        Lv = Lm @ v
        assert np.allclose(Lv, lam[l - 1, k - 1] * v, rtol=0, atol=1e-10 * np.abs(lam).max())
    assert np.allclose(O.alpha(nx, ny, dx, dy, 0.37), 0.37 * lam, rtol=1e-14, atol=0)


@pytest.mark.parametrize("nx,ny,y0,y1", [(8, 16, -1.0, 1.0), (16, 8, -0.5, 0.5),
                                         (16, 32, -0.5, 0.5)])
def test_poisson_matches_dense_direct_solve(nx, ny, y0, y1):
    """The 8x16 (7x15 = 105 unknowns) dense check of the sine solver, plus an
    anisotropic (dx != dy) and a transposed aspect ratio."""
    dx, dy = 1.0 / nx, (y1 - y0) / ny
    rhs = np.random.default_rng(6).normal(size=(ny - 1, nx - 1))
    ref = np.linalg.solve(dense_laplacian(nx, ny, dx, dy), rhs.ravel()).reshape(rhs.shape)
    got = O.poisson_solve(rhs, nx, ny, dx, dy)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("k,l", [(1, 1), (3, 2), (7, 13)])
def test_manufactured_discrete_modes(k, l):
    """rhs = lambda_kl sin(pi k i/nx) sin(pi l j/ny) returns the mode to
    1e-12 (the discrete-eigenvalue manufactured solution)."""
    nx, ny = 64, 128
    dx, dy = 1.0 / nx, 2.0 / ny
    i = np.arange(1, nx)
    j = np.arange(1, ny)
    mode = np.sin(np.pi * l * j / ny)[:, None] * np.sin(np.pi * k * i / nx)[None, :]
    Lm = dense_laplacian(nx, ny, dx, dy)
    rhs = (Lm @ mode.ravel()).reshape(mode.shape)        # lambda_kl * mode, built densely
    got = O.poisson_solve(rhs, nx, ny, dx, dy)
    assert np.linalg.norm(got - mode) <= 1e-12 * np.linalg.norm(mode)


def test_continuous_mode_second_order():
    """Against the continuous solution sin(k pi x) sin(l pi (y+1)/2) of
    lap(psi) = -pi^2 (k^2 + l^2/4) psi the error falls by ~4 per halving."""
    k, l = 2, 3
    errs = []
    for nx in (16, 32, 64, 128):
        ny = 2 * nx
        dx, dy = 1.0 / nx, 2.0 / ny
        x = np.arange(1, nx) * dx
        y = -1.0 + np.arange(1, ny) * dy
        exact = np.sin(l * np.pi * (y + 1) / 2)[:, None] * np.sin(k * np.pi * x)[None, :]
        rhs = -np.pi ** 2 * (k ** 2 + l ** 2 / 4.0) * exact
        got = O.poisson_solve(rhs, nx, ny, dx, dy)
        errs.append(np.max(np.abs(got - exact)))
    ratios = [errs[n] / errs[n + 1] for n in range(len(errs) - 1)]
    assert all(3.9 < r < 4.1 for r in ratios), ratios


def test_one_layer_scaling_by_Ro():
    """elliptic_one_layer solves Ro lap(psi) = Q."""
    nx, ny = 16, 32
    dx, dy = 1.0 / nx, 2.0 / ny
    Q = np.random.default_rng(8).normal(size=(ny - 1, nx - 1))
    Ro = 0.0016
    psi = O.elliptic_one_layer(Q, nx, ny, dx, dy, Ro)
    back = Ro * (dense_laplacian(nx, ny, dx, dy) @ psi.ravel()).reshape(Q.shape)
    assert np.linalg.norm(back - Q) <= 1e-12 * np.linalg.norm(Q)
