"""Gradient of a time-mean kinetic energy with respect to the wind-forcing
field, as a ``torch.autograd.Function`` over the library's tape and adjoint
calls (qg_tape_begin, qg_step, qg_energy_accumulate, qg_energy_gradient,
qg_adjoint_step).  The paper has no adjoint; the objective is the basin
kinetic energy of Section 5.2 averaged over a window of steps.

    J(F) = 1/(N - n0 + 1) * sum_{n = n0..N} E(psi^n),   psi^n = P^l S R^l w^n

All arithmetic runs in the library's kernels; this module only orders the
calls: a forward sweep that records the states and sums E on the device
(qg_energy_accumulate: no synchronisation per step), and a reverse sweep
that adds dE/dw at each time of the window and steps the adjoint back.
"""
from __future__ import annotations

import torch

from . import qg


class MeanKineticEnergy(torch.autograd.Function):
    """J = MeanKineticEnergy.apply(F, basin, w0, nsteps, first, every).

    F: forcing field (ny-1, nx-1) on the basin's device and dtype (the
    gradient is taken with respect to it); basin: a one-layer ``qg.Basin``;
    w0: the initial state; nsteps: N; first: n0; every: checkpoint interval
    of the tape (1 keeps every state).  Returns a 0-d float64 tensor on F's
    device."""

    @staticmethod
    def forward(ctx, F, basin, w0, nsteps: int, first: int, every: int = 1):
        h = basin.h
        basin.set_forcing(F)
        basin.set_state(w0)
        qg.qg_tape_begin(h, every, nsteps)
        K = nsteps - first + 1
        J = torch.zeros((), dtype=torch.float64, device=F.device)
        if first == 0:
            qg.qg_energy_accumulate(h, 1.0 / K, J)
        for n in range(1, nsteps + 1):
            basin.step(1)
            if n >= first:
                qg.qg_energy_accumulate(h, 1.0 / K, J)
        qg.qg_synchronize(h)
        ctx.basin, ctx.nsteps, ctx.first = basin, nsteps, first
        ctx.shape, ctx.dtype, ctx.device = F.shape, F.dtype, F.device
        return J

    @staticmethod
    def backward(ctx, grad_J):
        basin, N, n0 = ctx.basin, ctx.nsteps, ctx.first
        h = basin.h
        lam = torch.zeros(ctx.shape, dtype=ctx.dtype, device=ctx.device)
        gF = torch.zeros_like(lam)
        K = N - n0 + 1
        for n in range(N, 0, -1):
            if n >= n0:
                qg.qg_energy_gradient(h, 1.0 / K, lam)
            qg.qg_adjoint_step(h, 1, lam, gF)
        qg.qg_synchronize(h)
        qg.qg_tape_end(h)
        return grad_J.to(gF.dtype) * gF, None, None, None, None, None


def mean_kinetic_energy(F, basin, w0, nsteps: int, first: int, every: int = 1):
    return MeanKineticEnergy.apply(F, basin, w0, nsteps, first, every)
