"""Oracle of the scalar Poisson full-field inference problem (Sec. 3.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Forward problem, Eqs. (24)-(25): A U = F(theta) = M theta on the free nodes
and U = 0 on every boundary node.  A is the stiffness alpha int grad N_a .
grad N_b and M the mass matrix int N_a N_b, both from the element routine of
``fem_oracle.c``; the source is discretised by its nodal values theta.
Objective, Eq. (26): J(theta) = sum_{i in I_obs} (U(theta)[i] - U_obs[i])^2.
Gradient by the adjoint method of Sec. 3, Eqs. (17)-(23), with the
constraint C(U, theta) = A_f: U - M_f: theta (free rows) and U_c = 0:
    (A_ff)^T lambda_f = dJ/dU_f = 2 (U - U_obs) on the observed nodes,
    dJ/dtheta = -lambda^T dC/dtheta = (M_f:)^T lambda_f.
Optimiser: L-BFGS (scipy's L-BFGS-B), as the paper.  ``taylor_remainders``
gives the two residuals of Eqs. (27)-(28).  The linear steps use one sparse
LU factorisation of A_ff (the library routine ``scipy.sparse.linalg.splu``),
so no iterative tolerance enters the oracle.
"""
from __future__ import annotations

import ctypes

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import Mesh, lib, mesh


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def element_matrices(m: Mesh, alpha=1.0):
    """(Ke, Me), float64 [Ne, 8, 8]: element stiffness and mass (Eq. (25))."""
    Ke = np.zeros((m.n_cells, 8, 8))
    Me = np.zeros((m.n_cells, 8, 8))
    L = lib()
    for e in range(m.n_cells):
        L.oracle_poisson_element(_p(m.conn), _p(m.X), e, float(alpha), _p(Ke[e]), _p(Me[e]))
    return Ke, Me


def assemble(m: Mesh, alpha=1.0):
    """Global (A, M) as scipy CSR matrices, no boundary condition applied:
    the sum over cells of the element matrices (Algorithm 1, scalar)."""
    Ke, Me = element_matrices(m, alpha)
    r = np.repeat(m.conn.astype(np.int64), 8, axis=1).reshape(-1)
    c = np.tile(m.conn.astype(np.int64), (1, 8)).reshape(-1)
    n = m.n_nodes
    A = sp.coo_matrix((Ke.reshape(-1), (r, c)), shape=(n, n)).tocsr()
    M = sp.coo_matrix((Me.reshape(-1), (r, c)), shape=(n, n)).tocsr()
    return A, M


def apply(m: Mesh, alpha, x, mask=None):
    """y = A x matrix-free; masked nodes: x_c removed, y_c = x_c."""
    x = np.ascontiguousarray(x, np.float64).reshape(-1)
    y = np.zeros(m.n_nodes)
    mk = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    lib().oracle_poisson_apply(m.n_nodes, m.n_cells, _p(m.conn), _p(m.X), float(alpha), _p(x),
                               _p(mk), _p(y))
    return y


def load(m: Mesh, theta, mask=None):
    """F = M theta; F_c = 0 on masked nodes."""
    theta = np.ascontiguousarray(theta, np.float64).reshape(-1)
    F = np.zeros(m.n_nodes)
    mk = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    lib().oracle_poisson_load(m.n_nodes, m.n_cells, _p(m.conn), _p(m.X), _p(theta), _p(mk), _p(F))
    return F


class Problem:
    """The discretised constraint of Eq. (26) on mesh m with boundary mask
    (uint8 [N], 1 = u prescribed to 0), factorised once."""

    def __init__(self, m: Mesh, alpha, mask):
        self.m = m
        self.alpha = float(alpha)
        self.mask = np.ascontiguousarray(mask, np.uint8).reshape(-1)
        self.free = self.mask == 0
        self.A, self.M = assemble(m, alpha)
        self.Aff = self.A[self.free][:, self.free].tocsc()
        self.Mf = self.M[self.free]
        self.lu = spla.splu(self.Aff)

    def solve(self, theta):
        """U(theta): A_ff U_f = (M theta)_f, U_c = 0."""
        U = np.zeros(self.m.n_nodes)
        U[self.free] = self.lu.solve(self.Mf @ np.asarray(theta, np.float64))
        return U

    def objective(self, theta, obs, U_obs):
        U = self.solve(theta)
        d = U[obs] - U_obs
        return float(d @ d), U

    def gradient(self, theta, obs, U_obs):
        """(J, dJ/dtheta, U, lambda) by the adjoint method."""
        J, U = self.objective(theta, obs, U_obs)
        dJdU = np.zeros(self.m.n_nodes)
        dJdU[obs] = 2.0 * (U[obs] - U_obs)
        lam = np.zeros(self.m.n_nodes)
        lam[self.free] = self.lu.solve(dJdU[self.free], trans="T")
        g = self.Mf.T @ lam[self.free]
        return J, np.asarray(g).reshape(-1), U, lam

    def rel_l2_error(self, u_pred, u_true):
        """||u_pred - u_true||_L2 / ||u_true||_L2 with the L2 norm of the
        finite-element fields, ||v||^2 = v^T M v."""
        e = np.asarray(u_pred) - np.asarray(u_true)
        return float(np.sqrt(e @ (self.M @ e)) / np.sqrt(u_true @ (self.M @ u_true)))


def taylor_remainders(prob: Problem, theta, dtheta, obs, U_obs, hs):
    """r_zeroth(h) = |J(theta + h dtheta) - J(theta)| and
    r_first(h) = |J(theta + h dtheta) - J(theta) - h dJ/dtheta . dtheta|
    (Eqs. (27)-(28)) for each h in hs."""
    J0, g, _, _ = prob.gradient(theta, obs, U_obs)
    slope = float(g @ dtheta)
    r0, r1 = [], []
    for h in hs:
        Jh, _ = prob.objective(theta + h * dtheta, obs, U_obs)
        r0.append(abs(Jh - J0))
        r1.append(abs(Jh - J0 - h * slope))
    return np.array(r0), np.array(r1)


def infer(prob: Problem, obs, U_obs, theta0, maxiter=100, history=None):
    """The PDE-CO loop of Sec. 3 (forward solve, adjoint gradient, optimiser
    step) with L-BFGS-B as the optimiser.  Returns theta."""
    from scipy.optimize import minimize

    def fun(th):
        J, g, _, _ = prob.gradient(th, obs, U_obs)
        if history is not None:
            history.append(J)
        return J, g

    # the gradient entries scale with the cell volume, so the default
    # projected-gradient and relative-decrease stops would end the loop
    # after a few steps; only the iteration limit ends it here
    res = minimize(fun, np.asarray(theta0, np.float64), jac=True, method="L-BFGS-B",
                   options={"maxiter": maxiter, "gtol": 0.0, "ftol": 0.0})
    return res.x


def from_workload(w):
    """Mesh and Problem of an inputs.PoissonInference workload."""
    m = mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    return m, Problem(m, w.alpha, w.mask)
