"""torch.autograd.Function for x = D^-1 phi (Sec. 1: the inversions feed the
HMC fermion force).

forward:  x = D^-1 phi by the SAP-preconditioned FGCR of libqcdgb.
backward: for an upstream gradient g = dL/dx (torch convention
          dL/dRe + i dL/dIm), y = D^-+ g = g5 D^-1 g5 g (adjoint solve, a fresh
          Krylov space: the forward basis is not stored), then
            dL/dphi   = y,
            dL/dtheta = force(x, y) = -Re(y^+ dD/dtheta_a x)
          for the link deformation U_mu(x) -> exp(i theta_a lambda_a / 2) U_mu(x)
          at theta = 0 (theta has shape (V, 4, 8), float64).
All arithmetic runs in libqcdgb kernels; this module only moves tensors.
"""
from __future__ import annotations

import torch

from . import binding as B


class DiracSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, theta, lattice, params):
        x = torch.zeros_like(phi)
        B.qcd_solve(lattice.ctx, phi.contiguous(), x, 1, params)
        ctx.lattice = lattice
        ctx.params = params
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        lat, params = ctx.lattice, ctx.params
        g = g.contiguous()
        y = torch.zeros_like(g)
        B.qcd_solve_dagger(lat.ctx, g, y, params)  # y = D^-+ g = g5 D^-1 g5 g
        grad_theta = None
        if ctx.needs_input_grad[1]:
            grad_theta = torch.empty((lat.V, 4, 8), dtype=torch.float64, device=g.device)
            B.qcd_force(lat.ctx, x.contiguous(), y.contiguous(), grad_theta)
        return y, grad_theta, None, None


def dirac_solve(phi, theta, lattice, **solver_kw):
    """x = D^-1 phi, differentiable in phi and in the link parameters theta."""
    return DiracSolve.apply(phi, theta, lattice, B.solver_params(**solver_kw))
