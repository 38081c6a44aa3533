"""torch.autograd wrapper of the float64 fine run and its hand-written adjoint.

``fine_run_moments(U0, log_eps, ...)`` returns the conserved moments V(T) of
the lifted initial state U0 after ``nsteps`` upwind fine steps; its backward
calls ``pr_batch_adjoint`` (checkpointed recomputation, hand-written VJP of
each step), so gradients flow to the primitive initial state U0 and to
log(eps).  ``density_misfit`` builds the density-modes initial state
rho = 1 + a1 sin 2 pi x + a2 cos 4 pi x (u = 0, theta = 1) and returns the
L2 misfit sum_i (rho_i(T) - rho*_i)^2 dx.  Plumbing only: every numerical step
runs in libpr's CUDA kernels.
"""
from __future__ import annotations

import math

import numpy as np
import torch

import paper_2502_02704_gb300 as pr


class FineRunMoments(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, log_eps, geom):
        nx, nv, L, x0, x1, bc, dt, nsteps, ckpt = geom
        eps = math.exp(float(log_eps))
        inst = pr.instance(nx, nv, dt, L=L, x0=x0, x1=x1, bc=bc, eps=eps, scheme=pr.PR_UPWIND)
        b = pr.pr_batch_create([inst], pr.PR_FP64)
        try:
            U = U0.detach().to("cpu", torch.float64).numpy()
            pr.pr_batch_set_initial(b, 0, U)
            pr.pr_batch_run(b, nsteps)
            V = pr.pr_batch_moments(b, 0, pr.PR_CONSERVED)
        finally:
            pr.pr_batch_destroy(b)
        ctx.save_for_backward(U0.detach())
        ctx.geom = geom
        ctx.eps = eps
        return torch.as_tensor(V, dtype=torch.float64, device=U0.device)

    @staticmethod
    def backward(ctx, gV):
        (U0,) = ctx.saved_tensors
        nx, nv, L, x0, x1, bc, dt, nsteps, ckpt = ctx.geom
        inst = pr.instance(nx, nv, dt, L=L, x0=x0, x1=x1, bc=bc, eps=ctx.eps, scheme=pr.PR_UPWIND)
        b = pr.pr_batch_create([inst], pr.PR_FP64)
        try:
            pr.pr_batch_set_initial(b, 0, U0.to("cpu", torch.float64).numpy())
            dU0, de = pr.pr_batch_adjoint(b, 0, nsteps, gV.detach().to("cpu", torch.float64).numpy(), ckpt)
        finally:
            pr.pr_batch_destroy(b)
        return (torch.as_tensor(dU0, dtype=torch.float64, device=U0.device),
                torch.tensor(de, dtype=torch.float64), None)


def fine_run_moments(U0, log_eps, nx, nv, dt, nsteps, L=8.0, x0=0.0, x1=1.0, bc=pr.PR_BC_PERIODIC,
                     checkpoint=16):
    """Differentiable V(T) [5, nx] (conserved) of the upwind fine run from L(U0)."""
    return FineRunMoments.apply(U0, log_eps, (nx, nv, L, x0, x1, bc, dt, nsteps, checkpoint))


def density_modes_state(a1, a2, nx, device="cpu"):
    """Primitive state [5, nx] with rho = 1 + a1 sin 2 pi x + a2 cos 4 pi x, u = 0, theta = 1."""
    x = (torch.arange(nx, dtype=torch.float64, device=device) + 0.5) / nx
    rho = 1.0 + a1 * torch.sin(2 * math.pi * x) + a2 * torch.cos(4 * math.pi * x)
    z = torch.zeros_like(rho)
    return torch.stack([rho, z, z, z, torch.ones_like(rho)])


def density_misfit(a1, a2, log_eps, rho_target, nx, nv, dt, nsteps, L=8.0, checkpoint=16):
    """J = sum_i (rho_i(T) - rho*_i)^2 dx over periodic [0, 1)."""
    U0 = density_modes_state(a1, a2, nx, device=rho_target.device)
    V = fine_run_moments(U0, log_eps, nx, nv, dt, nsteps, L=L, checkpoint=checkpoint)
    return ((V[0] - rho_target) ** 2).sum() / nx
