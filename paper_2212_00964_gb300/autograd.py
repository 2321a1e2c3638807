"""torch.autograd.Function around fem_solve / fem_adjoint.

Forward: theta (per-cell parameter) -> u*(theta), the converged state of the
load-stepped Newton solve.  Only u* is saved (the checkpoint); no Newton or CG
iterate is stored.  Backward: the adjoint of Sec. 3, Eqs. (22)-(23),
dJ/dtheta = -lambda^T dC/dtheta with K(u*) lambda = dJ/du, computed by
fem_adjoint on the saved state.  Valid for path-independent (hyperelastic
or linear) laws, where the gradient depends only on the final state.
"""
from __future__ import annotations

import torch

from . import fem as F


class _SolveFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, solver):
        u = solver.forward_solve(theta.detach())
        ctx.solver = solver
        ctx.save_for_backward(theta.detach(), u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        theta, u = ctx.saved_tensors
        g = ctx.solver.adjoint(u, theta, grad_u.contiguous().to(torch.float64))
        return g.to(theta.dtype), None


class FemSolve:
    """Callable differentiable solve: ``u = FemSolve(mesh, mat, mask, u_bar)(theta)``."""

    def __init__(self, mesh, mat, mask, u_bar, f_ext=None, n_steps=1, options=None):
        self.mesh, self.mat, self.mask, self.u_bar = mesh, mat, mask, u_bar
        self.f_ext, self.n_steps = f_ext, n_steps
        self.options = options if options is not None else F.default_options()
        self.last_stats = None

    def forward_solve(self, theta):
        u = torch.zeros(self.mesh.n_dofs, dtype=torch.float64, device=theta.device)
        self.last_stats = F.fem_solve(self.mesh, self.mat, self.mask, self.u_bar, u, self.f_ext,
                                      theta.to(torch.float64).contiguous(), self.n_steps, self.options)
        return u

    def adjoint(self, u, theta, dJdu):
        g, st = F.fem_adjoint(self.mesh, self.mat, self.mask, u, dJdu, theta.to(torch.float64).contiguous(),
                              options=self.options)
        self.last_adjoint_stats = st
        return g

    def __call__(self, theta):
        return _SolveFn.apply(theta, self)
