"""Oracle of perfect J2 plasticity (Sec. 2.3, Eqs. (14)-(15)), small strain.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Every Gauss point carries the history of the previous load step: the total
strain eps^{k-1} and the stress sigma^{k-1}, float64 [Ne, 8, 3, 3] each.  At
load step k the prescribed DOFs take their step-k values and Newton solves
R(u^k; history) = 0 with the consistent tangent of the return map; the
linear step is ``scipy.sparse.linalg.spsolve`` on the free-free block of the
assembled tangent.  Once converged, the history becomes (eps^k, sigma^k).
Readings (the paper gives none of these): the Newton stop is
||R_free|| <= rtol * max(||R_free|| at iteration 0 of the step, sigma_y h^2),
h the smallest cell edge: the yield force of one cell face is the floor, so
a step with little or no load change, whose first residual is at the
rounding level of the internal forces, still ends; the first iterate of a
step is the previous converged state with the new prescribed values.
"""
from __future__ import annotations

import ctypes

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import Mesh, lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f(a, shape=None):
    a = np.ascontiguousarray(a, np.float64)
    return a if shape is None else a.reshape(shape)


class Material:
    def __init__(self, E, nu, sigma_y):
        self.E, self.nu, self.sy = float(E), float(nu), float(sigma_y)

    def args(self):
        return [self.E, self.nu, self.sy]


def zero_history(m: Mesh):
    return np.zeros((m.n_cells, 8, 3, 3)), np.zeros((m.n_cells, 8, 3, 3))


def stress(mat: Material, eps_old, sig_old, H):
    """(sigma^k, eps^k, f_yield) of one Gauss point (Eq. (15))."""
    sig = np.zeros(9)
    eps = np.zeros(9)
    f = lib().oracle_j2_stress(*mat.args(), _p(_f(eps_old, 9)), _p(_f(sig_old, 9)), _p(_f(H, 9)),
                               _p(sig), _p(eps))
    return sig.reshape(3, 3), eps.reshape(3, 3), f


def dstress(mat: Material, eps_old, sig_old, H, dH):
    dsig = np.zeros(9)
    lib().oracle_j2_dstress(*mat.args(), _p(_f(eps_old, 9)), _p(_f(sig_old, 9)), _p(_f(H, 9)),
                            _p(_f(dH, 9)), _p(dsig))
    return dsig.reshape(3, 3)


def gp_jxw(m: Mesh):
    """w_q det J per Gauss point, [Ne, 8]."""
    out = np.zeros((m.n_cells, 8))
    lib().oracle_gp_jxw(m.n_cells, _p(m.conn), _p(m.X), _p(out))
    return out


def residual(m: Mesh, mat: Material, hist, u, mask=None, f_ext=None):
    """(R, (eps^k, sigma^k), n_yield) at displacement u."""
    he, hs = (_f(h) for h in hist)
    u = _f(u).reshape(-1)
    R = np.zeros(m.n_dofs)
    eps = np.zeros((m.n_cells, 8, 3, 3))
    sig = np.zeros((m.n_cells, 8, 3, 3))
    mk = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    fe = None if f_ext is None else _f(f_ext)
    n = lib().oracle_j2_residual(m.n_nodes, m.n_cells, _p(m.conn), _p(m.X), *mat.args(), _p(he), _p(hs),
                                 _p(u), _p(fe), _p(mk), _p(R), _p(eps), _p(sig))
    return R, (eps, sig), int(n)


def tangent_apply(m: Mesh, mat: Material, hist, u, x, mask=None):
    he, hs = (_f(h) for h in hist)
    y = np.zeros(m.n_dofs)
    mk = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    lib().oracle_j2_tangent_apply(m.n_nodes, m.n_cells, _p(m.conn), _p(m.X), *mat.args(), _p(he), _p(hs),
                                  _p(_f(u).reshape(-1)), _p(_f(x).reshape(-1)), _p(mk), _p(y))
    return y


def assemble(m: Mesh, mat: Material, hist, u):
    """Global tangent (no boundary condition) as scipy CSR (Algorithm 1)."""
    he, hs = (_f(h) for h in hist)
    u = _f(u).reshape(-1)
    Ke = np.zeros((m.n_cells, 24, 24))
    L = lib()
    for e in range(m.n_cells):
        L.oracle_j2_element_tangent(_p(m.conn), _p(m.X), *mat.args(), _p(he), _p(hs), _p(u), e, _p(Ke[e]))
    dofs = (3 * m.conn.astype(np.int64)[:, :, None] + np.arange(3)[None, None, :]).reshape(m.n_cells, 24)
    r = np.repeat(dofs, 24, axis=1).reshape(-1)
    c = np.tile(dofs, (1, 24)).reshape(-1)
    return sp.coo_matrix((Ke.reshape(-1), (r, c)), shape=(m.n_dofs, m.n_dofs)).tocsr()


def newton_step(m: Mesh, mat: Material, hist, mask, u_bar, u0, rtol=1e-12, maxit=30):
    """Solve load step k: u_c = u_bar_c, R_free(u; hist) = 0.  Returns
    (u^k, new history, n_yield, iterations)."""
    mask = np.asarray(mask, np.uint8).reshape(-1)
    free = mask == 0
    u = np.array(u0, np.float64).reshape(-1)
    u[~free] = np.asarray(u_bar, np.float64).reshape(-1)[~free]
    h = min(m.lx / m.nx, m.ly / m.ny, m.lz / m.nz)
    ref = None
    for it in range(maxit + 1):
        R, new_hist, n_yield = residual(m, mat, hist, u, mask)
        nrm = float(np.linalg.norm(R))
        if ref is None:
            ref = max(nrm, mat.sy * h * h)
        if nrm <= rtol * ref:
            return u, new_hist, n_yield, it
        K = assemble(m, mat, hist, u)
        u[free] += spla.spsolve(K[free][:, free].tocsc(), -R[free])
    raise RuntimeError(f"J2 Newton: ||R|| = {nrm:.3e} after {maxit} iterations")


def solve_path(m: Mesh, mat: Material, mask, u_bars, rtol=1e-12):
    """Load path: one Newton solve per prescribed state in u_bars (list of
    [D] arrays).  Returns the list of (u^k, (eps^k, sigma^k), n_yield)."""
    hist = zero_history(m)
    u = np.zeros(m.n_dofs)
    out = []
    for ub in u_bars:
        u, hist, n_yield, _ = newton_step(m, mat, hist, mask, ub, u, rtol)
        out.append((u.copy(), hist, n_yield))
    return out


def volume_average(m: Mesh, field):
    """Volume average of a Gauss-point field [Ne, 8, ...]."""
    w = gp_jxw(m)
    return np.tensordot(w, field, axes=([0, 1], [0, 1])) / w.sum()
