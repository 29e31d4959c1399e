"""Independent constructions used by the oracle pins.

These build the 5-point Laplacian and the transfer operators as dense
matrices straight from their stencil definitions (Kronecker products of the
1-D second difference), so a test can compare the oracle's sine-transform
solver with a direct solve that shares none of its arithmetic.
"""
import numpy as np


def second_difference(n):
    """(n-1)x(n-1) matrix of u_{i-1} - 2u_i + u_{i+1} with u_0 = u_n = 0."""
    m = n - 1
    return (np.diag(-2.0 * np.ones(m)) + np.diag(np.ones(m - 1), 1)
            + np.diag(np.ones(m - 1), -1))


def dense_laplacian(nx, ny, dx, dy):
    """5-point Laplacian on the interior unknowns, flattened row-major [j, i]."""
    Ix, Iy = np.eye(nx - 1), np.eye(ny - 1)
    return (np.kron(Iy, second_difference(nx)) / dx ** 2
            + np.kron(second_difference(ny), Ix) / dy ** 2)


def node_coords(nx, ny, x0, x1, y0, y1):
    x = x0 + (x1 - x0) * np.arange(nx + 1) / nx
    y = y0 + (y1 - y0) * np.arange(ny + 1) / ny
    return np.meshgrid(x, y)  # X[j, i], Y[j, i]
