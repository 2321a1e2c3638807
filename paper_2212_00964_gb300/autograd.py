"""torch.autograd.Function around fem_solve / fem_adjoint, and around the
scalar Poisson solve of the full-field inference example (Sec. 3.1).

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


class _PoissonFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, solver):
        ctx.solver = solver
        return solver.forward_solve(theta.detach())

    @staticmethod
    def backward(ctx, grad_u):
        g = ctx.solver.adjoint(grad_u.contiguous().to(ctx.solver.dtype))
        return g, None


class PoissonSolve:
    """Differentiable theta -> u(theta) of the Poisson problem: A u = M theta
    on the free nodes, u = 0 on masked ones.  Backward: fem_poisson_adjoint
    (A lambda = dJ/du, dJ/dtheta = M lambda), so any torch objective of u
    gets its gradient by the adjoint method, as in the paper's PDE-CO loop."""

    def __init__(self, mesh, alpha=1.0, mask=None, rtol=None, maxit=10000, mixed=False, dtype=torch.float64):
        self.mesh, self.alpha, self.mask = mesh, float(alpha), mask
        self.rtol, self.maxit, self.mixed, self.dtype = rtol, maxit, mixed, dtype

    def forward_solve(self, theta):
        th = theta.to(self.dtype).contiguous()
        b = F.fem_poisson_apply(self.mesh, th, self.alpha, F.FEM_POISSON_MASS, self.mask)
        u, _, _ = F.fem_poisson_solve(self.mesh, b, self.alpha, self.mask, rtol=self.rtol, maxit=self.maxit,
                                      mixed=self.mixed)
        return u

    def adjoint(self, dJdu):
        g, _, _ = F.fem_poisson_adjoint(self.mesh, dJdu, self.alpha, self.mask, rtol=self.rtol, maxit=self.maxit,
                                        mixed=self.mixed)
        return g

    def __call__(self, theta):
        return _PoissonFn.apply(theta, self)
