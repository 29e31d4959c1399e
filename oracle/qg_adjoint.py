"""FP64 discrete adjoint of the one-layer CGPRK3 step (test infrastructure).

TEST INFRASTRUCTURE ONLY, like ``qg_oracle``: only the tests,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import it.

The paper has no adjoint.  This module differentiates the discrete step of
Section 3.2 exactly (it is the transpose of the step's Jacobian, not a
discretised continuous adjoint), for gradients of a time-mean kinetic
energy (Section 5.2) with respect to the wind-forcing field.

Derivation.  With psi = A w, A = P^l S R^l (restriction Eq. res l times, the
5-point Poisson solve S of Section 4.3, prolongation Eq. pro l times), the
right-hand side of one stage is
    G(w) = -J(A w, w) - (1/Ro) J(A w, y) + (1/Re) L w + F.
Its Jacobian applied to dw is
    -J(A dw, w) - J(psi, dw) - (1/Ro) J(A dw, y) + (1/Re) L dw.
With w, psi and every test field zero on the walls, three facts give the
transpose (each one is pinned in tests/test_oracle_adjoint.py):
  * K_p : b -> J(p, b) is skew-symmetric (Arakawa's enstrophy conservation,
    Section 4.1, polarised), and J(a, b) = -J(b, a) pointwise;
  * B : a -> J(a, y) is skew-symmetric (its closed form is a central x
    difference, skew, times a symmetric (1 4 1)/6 average in y);
  * A is symmetric: R = P^T/4 per level and S is the inverse of a symmetric
    matrix, so A^T = 4^-l P^l S 4^l R^l = A.
Hence
    G_w(w)^T lam = J(psi, lam) + (1/Re) L lam - A [J(w, lam) - (1/Ro) J(lam, y)].

The TVDRK3 step (Eq. TVDRK) in stage form w^(s+1) = a_s w^n + b_s (w^(s) +
dt G(w^(s))), (a, b) = (0, 1), (3/4, 1/4), (1/3, 2/3), is reversed stage by
stage: the adjoint of stage s sends lam_s to a_s lam_s (onto w^n) and to
b_s lam_s + b_s dt G_w(w^(s))^T lam_s (onto w^(s)), and adds b_s dt lam_s to
the forcing gradient (F enters G additively).
"""
from __future__ import annotations

import numpy as np

from . import qg_oracle as O

RK_A = (0.0, 0.75, 1.0 / 3.0)
RK_B = (1.0, 0.25, 2.0 / 3.0)


def _Y(b: O.Basin) -> np.ndarray:
    return np.repeat(O.grid_y(b)[:, None], b.nx + 1, axis=1)


def beta_jacobian(a: np.ndarray, b: O.Basin) -> np.ndarray:
    """J(a, y) at the interior nodes (Eq. ja1 with q = y); a is a node array."""
    return O.arakawa(a, _Y(b), b.dx, b.dy)


def rhs_adjoint(lam: np.ndarray, w: np.ndarray, psi: np.ndarray, b: O.Basin) -> np.ndarray:
    """G_w(w)^T lam (see the module docstring); lam, w, psi node arrays with
    zero walls, psi = A w.  Returns the interior array."""
    t = O.arakawa(w, lam, b.dx, b.dy) - beta_jacobian(lam, b) / b.Ro
    return (O.arakawa(psi, lam, b.dx, b.dy)
            + O.laplacian5(lam, b.dx, b.dy) / b.Re
            - O.interior(O.cgp_psi(O.embed(t), b)))


def stage_states(w: np.ndarray, b: O.Basin, F: np.ndarray | None = None):
    """w^(0) = w^n, w^(1), w^(2) of one CGPRK3 step and psi^(s) = A w^(s)
    (node arrays), the same arithmetic as ``qg_oracle.tvdrk3``."""
    ws, ps = [w], []
    for s in range(3):
        psi = O.cgp_psi(ws[s], b)
        ps.append(psi)
        if s < 2:
            G = O.rhs_omega(ws[s], psi, b, F)
            nxt = np.zeros_like(w)
            nxt[1:-1, 1:-1] = (RK_A[s] * O.interior(w)
                               + RK_B[s] * (O.interior(ws[s]) + b.dt * G))
            ws.append(nxt)
    return ws, ps


def adjoint_step(w: np.ndarray, lam: np.ndarray, b: O.Basin,
                 F: np.ndarray | None = None):
    """Transpose of one CGPRK3 step's Jacobian at the state w = w^n (node
    array).  lam is dJ/dw^(n+1) (interior array).  Returns (dJ/dw^n through
    this step, dJ/dF through this step), both interior arrays."""
    ws, ps = stage_states(w, b, F)
    lam_s = np.asarray(lam, dtype=np.float64)
    acc = np.zeros_like(lam_s)
    gF = np.zeros_like(lam_s)
    for s in (2, 1, 0):
        acc += RK_A[s] * lam_s
        gF += RK_B[s] * b.dt * lam_s
        back = RK_B[s] * lam_s + RK_B[s] * b.dt * rhs_adjoint(O.embed(lam_s), ws[s], ps[s], b)
        if s == 0:
            acc += back
        else:
            lam_s = back
    return acc, gF


def energy(w: np.ndarray, b: O.Basin) -> float:
    """E(A w): kinetic energy of the first-stage streamfunction of a state."""
    return O.kinetic_energy(O.cgp_psi(w, b), b.dx, b.dy)


def energy_gradient(w: np.ndarray, b: O.Basin) -> np.ndarray:
    """dE(A w)/dw at the interior nodes.  E(psi) = -1/2 dx dy sum psi L psi
    (summation by parts with psi = 0 on the walls), so dE/dpsi = -dx dy L psi
    and dE/dw = A^T(-dx dy L psi) = A(-dx dy L psi)."""
    psi = O.cgp_psi(w, b)
    t = -b.dx * b.dy * O.laplacian5(psi, b.dx, b.dy)
    return O.interior(O.cgp_psi(O.embed(t), b))


def _replace_forcing(b: O.Basin, F: np.ndarray) -> O.Basin:
    from dataclasses import replace
    return replace(b, forcing=np.asarray(F, dtype=np.float64))


def mean_energy(w0_int: np.ndarray, b: O.Basin, F: np.ndarray, nsteps: int,
                first: int) -> float:
    """J(F) = mean of E(A w^n) over n = first..nsteps, w^0 = w0, forcing F."""
    bf = _replace_forcing(b, F)
    w = O.embed(np.asarray(w0_int, dtype=np.float64))
    acc = energy(w, bf) if first == 0 else 0.0
    for n in range(1, nsteps + 1):
        w = O.cgprk3_step(w, bf)
        if n >= first:
            acc += energy(w, bf)
    return acc / (nsteps - first + 1)


def mean_energy_gradient(w0_int: np.ndarray, b: O.Basin, F: np.ndarray, nsteps: int,
                         first: int):
    """(J(F), dJ/dF) by a forward sweep that keeps every state and a reverse
    sweep of ``adjoint_step``."""
    bf = _replace_forcing(b, F)
    Fi = np.asarray(F, dtype=np.float64)
    K = nsteps - first + 1
    states = [O.embed(np.asarray(w0_int, dtype=np.float64))]
    for _ in range(nsteps):
        states.append(O.cgprk3_step(states[-1], bf))
    J = sum(energy(states[n], bf) for n in range(first, nsteps + 1)) / K
    lam = np.zeros_like(Fi)
    gF = np.zeros_like(Fi)
    for n in range(nsteps, 0, -1):
        if n >= first:
            lam = lam + energy_gradient(states[n], bf) / K
        lam, g = adjoint_step(states[n - 1], lam, bf, Fi)
        gF += g
    return J, gF
