"""torch.autograd bridge for the hand-written RKDG adjoint.

``RKDGSteps.apply(u0, solver, dt, nsteps, checkpoint_every)`` advances the
modal state u0 (a CPU float64 tensor (nc, nvar, np) in the user basis and
cell order) by nsteps fixed-dt SSP-RK3 steps with the solver's kernels and
returns u_N; its backward pass calls ``cswdg_adjoint_steps``, which reruns
the steps from u0 with checkpoints and sweeps back through the transposed
stage updates (operator and limiter, troubled-cell flags frozen as the
forward run set them) on the GPU.  dt > 0 is a fixed step size; dt <= 0
takes the CFL rule at every step, and the backward pass holds the step
sizes of that forward run fixed (their dependence on the state is not
differentiated).

``box_density_energy(uN, centroids, box)`` is the objective J of the
vortex gradient check: the integral of rho^2 over the cells whose centroid
lies in box, which in the physically orthonormal basis is the sum of the
squared density modes of those cells.
"""
from __future__ import annotations

import numpy as np
import torch


class RKDGSteps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, solver, dt, nsteps, checkpoint_every=20):
        u0n = u0.detach().cpu().numpy().astype(np.float64)
        t0 = solver.get_time()
        solver.write_modes(u0n)
        solver.step(dt, nsteps, 1e300)
        uN = solver.read_modes()
        ctx.solver, ctx.dt, ctx.nsteps, ctx.ck, ctx.t0 = solver, dt, nsteps, checkpoint_every, t0
        ctx.save_for_backward(u0.detach())
        return torch.from_numpy(uN).to(u0.dtype)

    @staticmethod
    def backward(ctx, gN):
        (u0,) = ctx.saved_tensors
        s = ctx.solver
        s.set_time(ctx.t0)
        _, g0 = s.adjoint_steps(u0.cpu().numpy().astype(np.float64), gN.detach().cpu().numpy().astype(np.float64),
                                ctx.dt, ctx.nsteps, ctx.ck)
        return torch.from_numpy(g0).to(u0.dtype), None, None, None, None


def box_density_energy(uN: torch.Tensor, centroids: np.ndarray, box) -> torch.Tensor:
    x0, x1, y0, y1 = box
    inside = (centroids[:, 0] > x0) & (centroids[:, 0] < x1) & (centroids[:, 1] > y0) & (centroids[:, 1] < y1)
    idx = torch.from_numpy(np.flatnonzero(inside))
    return (uN[idx, 0, :] ** 2).sum()
