"""Oracle of the topology-optimisation loop of Sec. 3.2 (SIMP compliance
minimisation under a volume constraint).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

One design iteration, as Sec. 3 lays out the PDE-CO loop:
  1. forward solve of the SIMP problem, Eqs. (29)-(30), with the per-cell
     density theta (``oracle.solve.linear_solve`` with the oracle's SIMP
     law E(theta) = E_min + theta^p (1 - E_min));
  2. compliance c = f . u (Eq. (31); for a nodal load vector f the boundary
     integral of u^h . t is f . U) and its gradient by the adjoint method
     (``oracle.solve.adjoint_gradient`` with dJ/du = f);
  3. the sensitivity filter: a convolution of the gradient with the cone
     kernel H_ef = max(0, r_min - |c_e - c_f|) (cell centres, in cell
     units), normalised by the kernel's row sums;
  4. one step of the method of moving asymptotes (Svanberg 1987) for
     min c(theta) s.t. mean(theta) - v_f <= 0, theta in [theta_min, 1].
An alternative optimiser step is the optimality-criteria update (``oc_step``);
``filter_transpose`` is the chain rule of the filter when it is applied to
the density instead of the sensitivities.
The MMA step follows Svanberg's 1987 construction, restated:
  * asymptotes: in the first two iterations L = x - s0 (x_max - x_min),
    U = x + s0 (x_max - x_min) with s0 = 0.5; afterwards each variable's
    distance to its asymptotes is scaled by 0.7 where its last two moves
    changed sign (oscillation), by 1.2 where they kept their sign, else 1;
  * move limits alpha = max(x_min, 0.9 L + 0.1 x), beta = min(x_max, 0.9 U + 0.1 x);
  * each function f_i (objective i = 0, constraint i = 1) is replaced by
    f~_i(y) = r_i + sum_j p_ij / (U_j - y_j) + q_ij / (x_j - L_j) ... with
    p_ij = (U_j - x_j)^2 max(df_i/dx_j, 0), q_ij = (x_j - L_j)^2 max(-df_i/dx_j, 0)
    and r_i chosen so that f~_i(x) = f_i(x);
  * the convex separable subproblem min f~_0 s.t. f~_1 <= 0, alpha <= y <= beta
    is solved through its one-dimensional dual: for a multiplier lam >= 0
    each y_j minimises (p_0j + lam p_1j)/(U_j - y) + (q_0j + lam q_1j)/(y - L_j)
    in closed form (clipped to [alpha_j, beta_j]); lam = 0 if that point is
    feasible, else the root of f~_1(y(lam)) = 0 by bisection (f~_1(y(lam))
    is non-increasing in lam).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import Material, Mesh
from . import solve as osolve


def filter_matrix(nx, ny, nz, rmin):
    """Cone-kernel weights H (Ne x Ne, CSR) between cell centres within
    distance r_min (in cell units); cell id = i + nx (j + ny k)."""
    rows, cols, vals = [], [], []
    R = int(np.ceil(rmin)) - 1
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                e = i + nx * (j + ny * k)
                for kk in range(max(0, k - R), min(nz, k + R + 1)):
                    for jj in range(max(0, j - R), min(ny, j + R + 1)):
                        for ii in range(max(0, i - R), min(nx, i + R + 1)):
                            di, dj, dk = ii - i, jj - j, kk - k
                            w = rmin - np.sqrt(di * di + dj * dj + dk * dk)
                            if w > 0:
                                rows.append(e)
                                cols.append(ii + nx * (jj + ny * kk))
                                vals.append(w)
    n = nx * ny * nz
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def filter_sensitivities(H, g):
    """g~_e = sum_f H_ef g_f / sum_f H_ef."""
    return (H @ g) / np.asarray(H.sum(axis=1)).reshape(-1)


def filter_transpose(H, g):
    """The transpose of the normalised filter: (diag(1/Hs) H)^T g =
    H^T (g / Hs), Hs the row sums.  With the filter applied to the density
    (theta~ = filter(theta) enters the physics) this carries dJ/dtheta~ back
    to dJ/dtheta by the chain rule."""
    hs = np.asarray(H.sum(axis=1)).reshape(-1)
    return H.T @ (g / hs)


def oc_step(x, g, dv, volfrac, move=0.2, x_min=0.0, x_max=1.0):
    """One optimality-criteria update for min c(x) s.t. sum dv x <= volfrac
    sum dv (the classic SIMP update; an alternative to MMA).  With
    B_e(lam) = -g_e / (lam dv_e) (g <= 0 for compliance):
        x_new = clip(x B^(1/2), max(x_min, x - move), min(x_max, x + move)),
    lam found by bisection on the volume, which is non-increasing in lam
    (on log(lam), until the bracket's relative width is 1e-13 or after 200
    halvings).  Returns (x_new, lam)."""
    x = np.asarray(x, np.float64)
    g = np.minimum(np.asarray(g, np.float64), 0.0)
    dv = np.asarray(dv, np.float64)
    target = volfrac * dv.sum()
    lo_b = np.maximum(x_min, x - move)
    hi_b = np.minimum(x_max, x + move)

    def x_of(lam):
        return np.clip(x * np.sqrt(-g / (lam * dv)), lo_b, hi_b)

    lo, hi = 1e-40, 1e40
    for _ in range(200):
        mid = np.sqrt(lo * hi)
        if (dv @ x_of(mid)) > target:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-13 * hi:
            break
    return x_of(hi), hi


class MMA:
    """Method of moving asymptotes for one inequality constraint f1 <= 0."""

    def __init__(self, n, x_min, x_max, s0=0.5, s_dec=0.7, s_inc=1.2):
        self.x_min = np.broadcast_to(np.asarray(x_min, np.float64), (n,)).copy()
        self.x_max = np.broadcast_to(np.asarray(x_max, np.float64), (n,)).copy()
        self.s0, self.s_dec, self.s_inc = s0, s_dec, s_inc
        self.k = 0
        self.x1 = self.x2 = self.L = self.U = None
        self.lam = 0.0

    def _asymptotes(self, x):
        span = self.x_max - self.x_min
        if self.k < 2:
            L = x - self.s0 * span
            U = x + self.s0 * span
        else:
            sgn = (x - self.x1) * (self.x1 - self.x2)
            fac = np.where(sgn < 0, self.s_dec, np.where(sgn > 0, self.s_inc, 1.0))
            L = x - fac * (self.x1 - self.L)
            U = x + fac * (self.U - self.x1)
        return L, U

    def step(self, x, f0, df0, f1, df1):
        x = np.asarray(x, np.float64)
        L, U = self._asymptotes(x)
        alpha = np.maximum(self.x_min, 0.9 * L + 0.1 * x)
        beta = np.minimum(self.x_max, 0.9 * U + 0.1 * x)
        dU, dL = U - x, x - L
        p0 = dU ** 2 * np.maximum(df0, 0.0)
        q0 = dL ** 2 * np.maximum(-df0, 0.0)
        p1 = dU ** 2 * np.maximum(df1, 0.0)
        q1 = dL ** 2 * np.maximum(-df1, 0.0)
        r1 = f1 - np.sum(p1 / dU + q1 / dL)

        def y_of(lam):
            P = p0 + lam * p1
            Q = q0 + lam * q1
            sP, sQ = np.sqrt(P), np.sqrt(Q)
            den = sP + sQ
            # P = Q = 0: the variable enters neither function; stay at x
            y = np.where(den > 0, (sP * L + sQ * U) / np.where(den > 0, den, 1.0), x)
            return np.clip(y, alpha, beta)

        def g1(lam):
            y = y_of(lam)
            return r1 + np.sum(p1 / (U - y) + q1 / (y - L))

        lam = 0.0
        if g1(0.0) > 0:
            lo, hi = 0.0, 1.0
            while g1(hi) > 0:
                lo, hi = hi, 2.0 * hi
                if hi > 1e300:
                    raise RuntimeError("MMA: no feasible multiplier")
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if mid == lo or mid == hi:
                    break
                if g1(mid) > 0:
                    lo = mid
                else:
                    hi = mid
            lam = hi
        y = y_of(lam)
        self.x2, self.x1 = self.x1, x.copy()
        self.L, self.U = L, U
        self.lam = lam
        self.k += 1
        return y


def compliance_and_gradient(m: Mesh, mat: Material, mask, f, theta, pattern=None):
    """(c, dc/dtheta, u) of the SIMP cantilever at density theta."""
    ubar = np.zeros(m.n_dofs)
    u = osolve.linear_solve(m, mat, mask, ubar, f, theta, pattern)
    g, _ = osolve.adjoint_gradient(m, mat, mask, u, f, theta, pattern=pattern)
    return float(f @ u), g, u


def simp_scale(theta, p=3.0, emin=1e-3):
    """(s, ds/dtheta) of the SIMP law s = emin + theta^p (1 - emin)."""
    theta = np.asarray(theta, np.float64)
    return emin + theta ** p * (1 - emin), p * theta ** (p - 1) * (1 - emin)


def compliance_and_gradient_nh(m: Mesh, E, nu, mask, f, theta, p=3.0, emin=1e-3, n_steps=1, pattern=None,
                               rtol=1e-12):
    """(c, dc/dtheta, u) for SIMP applied to the Neo-Hookean law, the
    paper's plate (Eqs. (29)-(30): theta^p P): the per-cell stiffness scale
    is s(theta) (both moduli scale with E, so s P(F; E) = P(F; s E)); the
    adjoint gives dc/ds, and dc/dtheta = dc/ds ds/dtheta."""
    mat = Material(2, E, nu)
    s, ds = simp_scale(theta, p, emin)
    u = osolve.newton_solve(m, mat, mask, np.zeros(m.n_dofs), f, s, n_steps=n_steps, pattern=pattern, rtol=rtol)
    g_s, _ = osolve.adjoint_gradient(m, mat, mask, u, f, s, pattern=pattern)
    return float(f @ u), g_s * ds, u


def optimise(m: Mesh, mat: Material, mask, f, volfrac=0.5, rmin=1.5, n_iter=30, theta_min=0.0,
             history=None):
    """The design loop (steps 1-4 above) from the uniform design theta =
    volfrac.  Returns theta; appends (c, mean theta) per iteration to
    history."""
    theta = np.full(m.n_cells, float(volfrac))
    H = filter_matrix(m.nx, m.ny, m.nz, rmin)
    mma = MMA(m.n_cells, theta_min, 1.0)
    pattern = osolve._pattern(m)
    for _ in range(n_iter):
        c, g, _ = compliance_and_gradient(m, mat, mask, f, theta, pattern)
        if history is not None:
            history.append((c, float(theta.mean())))
        gf = filter_sensitivities(H, g)
        theta = mma.step(theta, c, gf, float(theta.mean() - volfrac),
                         np.full(m.n_cells, 1.0 / m.n_cells))
    return theta
