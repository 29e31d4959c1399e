"""Seeded synthetic inputs shared by the tests, the benchmark and users.

This module holds no arithmetic of the method: it only draws numbers.  Every
generator takes an explicit seed and returns float64 numpy arrays in the
exchange layout of the C-ABI, an interior array of shape (ny-1, nx-1),
row-major, x fastest.  Random numbers are drawn with numpy's PCG64
(``numpy.random.default_rng``).
"""
from __future__ import annotations

import numpy as np

__all__ = ["perturbation", "smooth_field", "random_field", "gyre_state",
           "perturbed_forcing_field"]


def random_field(nx: int, ny: int, seed: int, std: float = 1.0) -> np.ndarray:
    """i.i.d. N(0, std^2) values on the interior nodes."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, std, size=(ny - 1, nx - 1))


def perturbation(nx: int, ny: int, seed: int, var: float = 1e-2) -> np.ndarray:
    """The seeded initial perturbation: i.i.d. N(0, var) interior vorticity
    (variance ``var``, so the standard deviation is sqrt(var))."""
    return random_field(nx, ny, seed, std=float(np.sqrt(var)))


def smooth_field(nx: int, ny: int, seed: int, nmodes: int = 6,
                 amp: float = 1.0, noise: float = 0.0) -> np.ndarray:
    """A sum of ``nmodes`` x ``nmodes`` low sine modes with N(0, amp^2)
    coefficients scaled by 1/(k l), plus optional N(0, noise^2) noise."""
    rng = np.random.default_rng(seed)
    x = np.arange(1, nx) / nx
    y = np.arange(1, ny) / ny
    out = np.zeros((ny - 1, nx - 1))
    for k in range(1, nmodes + 1):
        for l in range(1, nmodes + 1):
            c = rng.normal(0.0, amp) / (k * l)
            out += c * np.sin(np.pi * l * y)[:, None] * np.sin(np.pi * k * x)[None, :]
    if noise:
        out += rng.normal(0.0, noise, size=out.shape)
    return out


def gyre_state(nx: int, ny: int, seed: int, amp: float = 200.0,
               var: float = 1e-2) -> np.ndarray:
    """A stand-in for a spun-up double-gyre vorticity field: a smooth
    four-cell pattern with a western-boundary concentration and random
    mesoscale modes, plus N(0, var) noise.  Only its shape and magnitude
    matter (it is used where throughput, not the trajectory, is measured)."""
    rng = np.random.default_rng(seed)
    x = (np.arange(1, nx) / nx)[None, :]
    y = (np.arange(1, ny) / ny)[:, None]
    west = np.exp(-x / 0.05)
    field = amp * west * np.sin(2.0 * np.pi * y) + 0.2 * amp * np.sin(np.pi * x) * np.sin(4.0 * np.pi * y)
    for _ in range(12):
        k, l = rng.integers(2, 24, size=2)
        field += rng.normal(0.0, 0.05 * amp) * np.sin(np.pi * k * x) * np.sin(np.pi * l * y)
    field += rng.normal(0.0, np.sqrt(var), size=field.shape)
    return field


def perturbed_forcing_field(nx: int, ny: int, seed: int, Ro: float,
                            y0: float = -1.0, y1: float = 1.0,
                            nmodes: int = 8, amp: float = 0.05) -> np.ndarray:
    """sin(pi y)/Ro on the interior nodes plus a seeded smooth perturbation:
    a sum of ``nmodes`` low sine modes with N(0, amp^2) coefficients, scaled
    by 1/Ro."""
    rng = np.random.default_rng(seed)
    y = y0 + (y1 - y0) * np.arange(1, ny) / ny
    base = np.repeat((np.sin(np.pi * y) / Ro)[:, None], nx - 1, axis=1)
    xs = np.arange(1, nx) / nx
    ys = np.arange(1, ny) / ny
    pert = np.zeros_like(base)
    for _ in range(nmodes):
        k, l = rng.integers(1, 5, size=2)
        pert += rng.normal(0.0, amp) * np.sin(np.pi * k * xs)[None, :] * np.sin(np.pi * l * ys)[:, None]
    return base + pert / Ro


def unit_directions(nx: int, ny: int, count: int, seed: int) -> np.ndarray:
    """`count` seeded random fields of unit root-mean-square value, each an
    interior array (ny - 1, nx - 1): directions for directional derivatives
    with respect to a field."""
    rng = np.random.default_rng(seed)
    out = rng.normal(size=(count, ny - 1, nx - 1))
    rms = np.sqrt(np.mean(out * out, axis=(1, 2)))
    return out / rms[:, None, None]
