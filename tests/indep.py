"""Independent formulations used to pin the oracle (test-only, numpy).

Each function here computes a quantity the oracle also computes, but by a
different route, so that a dropped term, a wrong sign or a transposed
operand in the oracle shows up as a mismatch:
  * ``voigt_ke``: linear-elastic element stiffness by the engineering
    B-matrix / Voigt D-matrix formulation (the oracle uses the tensor form
    sigma : grad phi with JVPs);
  * ``nh_energy``: the Neo-Hookean strain energy W(F) typed from Sec. 2.3,
    Eq. (13) of the paper (the oracle only has P = dW/dF and dP);
  * rigid-body modes, face-load weights and the uniaxial closed form;
  * ``hex_volume``: cell volume by a 3-point Gauss rule of det J.
"""
from __future__ import annotations

import numpy as np

# VTK hexahedron corner signs (reference coordinates)
CORNERS = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                    [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], float)


def lame(E, nu):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def voigt_D(E, nu):
    lam, mu = lame(E, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3:, 3:] = np.eye(6 - 3) * mu
    return D


def box_grad(hx, hy, hz, xi):
    """Physical shape gradients of an axis-aligned box cell at reference xi."""
    s = CORNERS
    f = 1 + s * np.asarray(xi)[None, :]
    g = np.zeros((8, 3))
    g[:, 0] = s[:, 0] * f[:, 1] * f[:, 2] / 8 * (2 / hx)
    g[:, 1] = f[:, 0] * s[:, 1] * f[:, 2] / 8 * (2 / hy)
    g[:, 2] = f[:, 0] * f[:, 1] * s[:, 2] / 8 * (2 / hz)
    return g


def voigt_ke(hx, hy, hz, E, nu):
    """K_e = sum_q B^T D B detJ, Voigt order (xx, yy, zz, yz, xz, xy),
    engineering shear strains; DOF order 3a+i."""
    D = voigt_D(E, nu)
    g1 = 1 / np.sqrt(3)
    Ke = np.zeros((24, 24))
    detJ = hx * hy * hz / 8
    for c in (-g1, g1):
        for b in (-g1, g1):
            for a in (-g1, g1):
                G = box_grad(hx, hy, hz, (a, b, c))
                B = np.zeros((6, 24))
                for n in range(8):
                    dx, dy, dz = G[n]
                    B[0, 3 * n] = dx
                    B[1, 3 * n + 1] = dy
                    B[2, 3 * n + 2] = dz
                    B[3, 3 * n + 1] = dz
                    B[3, 3 * n + 2] = dy
                    B[4, 3 * n] = dz
                    B[4, 3 * n + 2] = dx
                    B[5, 3 * n] = dy
                    B[5, 3 * n + 1] = dx
                Ke += B.T @ D @ B * detJ
    return Ke


def rigid_modes(X):
    """6 infinitesimal rigid-body modes of nodal coordinates X [n,3] -> [6, 3n]."""
    n = X.shape[0]
    modes = []
    for i in range(3):
        m = np.zeros((n, 3))
        m[:, i] = 1
        modes.append(m.reshape(-1))
    for axis in range(3):
        w = np.zeros(3)
        w[axis] = 1
        modes.append(np.cross(w[None, :], X).reshape(-1))
    return np.array(modes)


def nh_energy(F, E, nu):
    """W(F) = G/2 (J^{-2/3} I1 - 3) + kappa/2 (J - 1)^2, Eq. (13)."""
    G = E / (2 * (1 + nu))
    kappa = E / (3 * (1 - 2 * nu))
    J = np.linalg.det(F)
    I1 = np.trace(F.T @ F)
    return G / 2 * (J ** (-2 / 3) * I1 - 3) + kappa / 2 * (J - 1) ** 2


def fd_grad(fun, x, h=1e-6):
    x = np.array(x, float)
    g = np.zeros_like(x)
    it = np.nditer(x, flags=["multi_index"])
    for _ in it:
        idx = it.multi_index
        xp = x.copy()
        xm = x.copy()
        xp[idx] += h
        xm[idx] -= h
        g[idx] = (fun(xp) - fun(xm)) / (2 * h)
    return g


def hex_volume(Xe):
    """Volume of a trilinear hexahedron with corners Xe [8, 3] (VTK order):
    the integral of det(dX/dxi) over [-1, 1]^3 by a 3-point Gauss-Legendre
    rule per axis (det J is at most quadratic in each reference coordinate,
    so the rule is exact)."""
    pts, wts = np.polynomial.legendre.leggauss(3)
    s = CORNERS
    vol = 0.0
    for a, wa in zip(pts, wts):
        for b, wb in zip(pts, wts):
            for c, wc in zip(pts, wts):
                p = np.array([a, b, c])
                f = 1 + s * p[None, :]
                dN = np.stack([s[:, 0] * f[:, 1] * f[:, 2], f[:, 0] * s[:, 1] * f[:, 2],
                               f[:, 0] * f[:, 1] * s[:, 2]], axis=1) / 8
                vol += wa * wb * wc * np.linalg.det(Xe.T @ dN)
    return vol


def random_rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def face_weight_closed_form(nx, ny, nz, lx, ly, lz, face, t):
    """Exact nodal forces of a uniform traction on an axis-aligned box face:
    each face node gets t * (cell face area) * (number of adjacent face cells)/4."""
    D = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    f = np.zeros(D)
    n = [nx, ny, nz]
    L = [lx, ly, lz]
    d = "xyz".index(face[0])
    side = int(face[1])
    d1, d2 = (d + 1) % 3, (d + 2) % 3
    area = (L[d1] / n[d1]) * (L[d2] / n[d2])
    for a in range(n[d1] + 1):
        for b in range(n[d2] + 1):
            ca = 1 + (0 < a < n[d1])
            cb = 1 + (0 < b < n[d2])
            idx = [0, 0, 0]
            idx[d] = n[d] if side else 0
            idx[d1] = a
            idx[d2] = b
            node = idx[0] + (nx + 1) * (idx[1] + (ny + 1) * idx[2])
            f[3 * node:3 * node + 3] += np.asarray(t) * area * ca * cb / 4
    return f
