"""Oracle drivers: Newton with load stepping, linear solve, adjoint gradient.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Newton follows Sec. 2.1, Eq. (4): at the current u solve the linearised
problem K(u) du = -R(u) for the free DOFs and update.  The linear step is the
library routine ``scipy.sparse.linalg.spsolve`` on the free-free block of the
oracle-assembled tangent (Algorithm 1), so no iterative-solver tolerance
enters the oracle.  Readings (the paper gives none of these):
  * load steps: S uniform increments; at step s the prescribed DOFs are set to
    (s/S) * u_bar and the free DOFs start from the previous converged state;
  * convergence: ||R_free||_2 <= rtol * ||R_free||_2 of the first iteration of
    step 1 (rtol 1e-12), at most 50 iterations, else not converged;
  * det F <= 0 at any Gauss point marks an inverted state.
The adjoint follows Sec. 3, Eqs. (22)-(23): K(u*)^T lambda = dJ/du on the
free DOFs (lambda_c = 0), then dJ/dtheta = -lambda^T dC/dtheta + dJ/dtheta|explicit.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import Material, Mesh, assemble, csr, residual, scatter_map, vjp


class NotConverged(RuntimeError):
    pass


class Inverted(RuntimeError):
    pass


def _pattern(m: Mesh):
    row_ptr, col = csr(m)
    return row_ptr, col, scatter_map(m, row_ptr, col)


def newton_solve(m: Mesh, mat: Material, mask, u_bar, f_ext=None, cell_param=None,
                 n_steps=1, rtol=1e-12, maxit=50, u0=None, pattern=None, history=None):
    """Solve R_free(u) = 0 with u_c = u_bar_c (prescribed), load-stepped.

    mask: uint8 [D] (1 = prescribed); u_bar: float64 [D] final prescribed
    values (only masked entries are read); f_ext: float64 [D] or None.
    Returns u (float64 [D]).
    """
    mask = np.asarray(mask, np.uint8).reshape(-1)
    free = mask == 0
    u_bar = np.asarray(u_bar, np.float64).reshape(-1)
    u = np.zeros(m.n_dofs) if u0 is None else np.array(u0, np.float64).reshape(-1)
    if pattern is None:
        pattern = _pattern(m)
    r_ref = None
    for s in range(1, n_steps + 1):
        u[~free] = (s / n_steps) * u_bar[~free]
        for it in range(maxit + 1):
            R, jmin = residual(m, mat, u, cell_param, f_ext, mask, return_jmin=True)
            if jmin <= 0.0:
                raise Inverted(f"det F = {jmin} <= 0 at step {s}, iteration {it}")
            nrm = float(np.linalg.norm(R))
            if r_ref is None:
                r_ref = nrm if nrm > 0 else 1.0
            if history is not None:
                history.append((s, it, nrm))
            if nrm <= rtol * r_ref:
                break
            if it == maxit:
                raise NotConverged(f"step {s}: ||R|| = {nrm:.3e} after {maxit} iterations")
            K = assemble(m, mat, u, cell_param, None, pattern)
            Kff = K[free][:, free].tocsc()
            u[free] += spla.spsolve(Kff, -R[free])
    return u


def linear_solve(m: Mesh, mat: Material, mask, u_bar, f_ext=None, cell_param=None, pattern=None):
    """One exact Newton step from u = u_bar on the prescribed DOFs: the
    solution of the linear problem for linear elasticity / SIMP."""
    mask = np.asarray(mask, np.uint8).reshape(-1)
    free = mask == 0
    u = np.zeros(m.n_dofs)
    u[~free] = np.asarray(u_bar, np.float64).reshape(-1)[~free]
    if pattern is None:
        pattern = _pattern(m)
    R = residual(m, mat, u, cell_param, f_ext, mask)
    K = assemble(m, mat, u, cell_param, None, pattern)
    u[free] += spla.spsolve(K[free][:, free].tocsc(), -R[free])
    return u


def adjoint_gradient(m: Mesh, mat: Material, mask, u_star, dJdu, cell_param=None,
                     dJdtheta=None, pattern=None):
    """dJ/dtheta (per cell) at the converged state u_star (Eqs. (22)-(23))."""
    mask = np.asarray(mask, np.uint8).reshape(-1)
    free = mask == 0
    if pattern is None:
        pattern = _pattern(m)
    K = assemble(m, mat, u_star, cell_param, None, pattern)
    lam = np.zeros(m.n_dofs)
    rhs = np.asarray(dJdu, np.float64).reshape(-1)[free]
    lam[free] = spla.spsolve(K[free][:, free].T.tocsc(), rhs)
    g = vjp(m, mat, u_star, lam, cell_param, mask)
    if dJdtheta is not None:
        g = g + np.asarray(dJdtheta, np.float64)
    return g, lam
