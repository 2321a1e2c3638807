"""Pins of the oracle's solves and gradients: manufactured-solution convergence
rates, homogeneous uniaxial Neo-Hookean closed form, the c0 linear solve
against an independent assembly, the self-adjoint SIMP compliance gradient in
closed form, central finite differences and the Taylor test of Sec. 3.1
(Eqs. (27)-(28))."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from oracle import solve as osolve
from paper_2212_00964_gb300 import inputs
from tests import indep

# ---------------------------------------------------------------- MMS ------
AMP = np.array([[1.0, 0.7, 0.5], [0.6, 1.1, 0.4], [0.3, 0.8, 0.9]])
PH = np.array([[0.1, 0.4, 0.2], [0.3, 0.0, 0.5], [0.6, 0.2, 0.1]])
FREQ = np.pi * np.array([[1.0, 1.0, 0.5], [0.5, 1.0, 1.0], [1.0, 0.5, 1.0]])


def u_exact(x):
    """u_i = AMP_i0 * prod_j sin(FREQ_ij x_j + PH_ij); x [..., 3]."""
    out = np.empty(x.shape)
    for i in range(3):
        out[..., i] = AMP[i, 0] * np.prod(np.sin(FREQ[i] * x + PH[i]), axis=-1)
    return out


def grad_exact(x):
    g = np.empty(x.shape + (3,))
    for i in range(3):
        s = np.sin(FREQ[i] * x + PH[i])
        c = np.cos(FREQ[i] * x + PH[i])
        for k in range(3):
            fac = np.ones(x.shape[:-1])
            for j in range(3):
                fac = fac * (FREQ[i, j] * c[..., j] if j == k else s[..., j])
            g[..., i, k] = AMP[i, 0] * fac
    return g


def body_force_exact(x, E, nu, h=1e-4):
    """b = -div sigma(u_exact), divergence by central differences of the
    analytic stress (error O(h^2) ~ 1e-7, far below the discretisation error)."""
    lam, mu = indep.lame(E, nu)

    def sigma(xx):
        H = grad_exact(xx)
        eps = 0.5 * (H + np.swapaxes(H, -1, -2))
        tr = np.trace(eps, axis1=-2, axis2=-1)
        return lam * tr[..., None, None] * np.eye(3) + 2 * mu * eps

    b = np.zeros(x.shape)
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        b -= (sigma(x + e)[..., :, j] - sigma(x - e)[..., :, j]) / (2 * h)
    return b


def mms_errors(n):
    E, nu = 1.0, 0.3
    m = oracle.mesh(n, n, n)
    mat = oracle.Material(oracle.LINEAR, E, nu)
    specs = [(f, c, 0.0) for f in ("x0", "x1", "y0", "y1", "z0", "z1") for c in range(3)]
    mask, _ = inputs.dirichlet(n, n, n, specs)
    ubar = u_exact(m.X).reshape(-1)
    xg = oracle.gauss_points_phys(m)
    f = oracle.body_force(m, body_force_exact(xg, E, nu))
    u = osolve.linear_solve(m, mat, mask, ubar, f)
    # errors at the Gauss points
    gp, w = oracle.gauss()
    h = 1.0 / n
    detJ = h ** 3 / 8
    U = u.reshape(-1, 3)[m.conn]  # [Ne, 8, 3]
    e2 = 0.0
    g2 = 0.0
    for q in range(8):
        N, _ = oracle.shape(*gp[q])
        G = indep.box_grad(h, h, h, gp[q])
        uh = np.einsum("a,eai->ei", N, U)
        gh = np.einsum("eai,aj->eij", U, G)
        e2 += w[q] * detJ * np.sum((uh - u_exact(xg[:, q])) ** 2)
        g2 += w[q] * detJ * np.sum((gh - grad_exact(xg[:, q])) ** 2)
    return np.sqrt(e2), np.sqrt(g2)


def test_mms_convergence_rates():
    errs = [mms_errors(n) for n in (4, 8, 16)]
    l2 = [e[0] for e in errs]
    h1 = [e[1] for e in errs]
    r_l2 = np.log2(l2[1] / l2[2])
    r_h1 = np.log2(h1[1] / h1[2])
    assert 1.9 <= r_l2 <= 2.1, (l2, r_l2)
    assert 0.9 <= r_h1 <= 1.1, (h1, r_h1)


# ------------------------------------------------- uniaxial closed form ----
def test_nh_homogeneous_uniaxial_closed_form():
    """Roller BCs (u_x=0 on x=0, u_y=0 on y=0, u_z=0 on z=0) and u_x=delta on
    x=1 make the exact solution affine: F = diag(1+delta, l2, l2) with l2 from
    P_yy = 0 (P from the energy W of Eq. (13), by differentiation in the test)."""
    E, nu, delta = 10.0, 0.3, -0.1
    n = 3
    m = oracle.mesh(n, n, n)
    mat = oracle.Material(oracle.NEOHOOKE, E, nu)
    mask, ubar = inputs.dirichlet(n, n, n, [("x0", 0, 0.0), ("y0", 1, 0.0), ("z0", 2, 0.0),
                                            ("x1", 0, delta)])
    u = osolve.newton_solve(m, mat, mask, ubar, n_steps=2)

    l1 = 1 + delta

    def pyy(l2):
        F = np.diag([l1, l2, l2])
        return indep.fd_grad(lambda Fm: indep.nh_energy(Fm, E, nu), F, h=1e-6)[1, 1]

    lo, hi = 0.8, 1.5
    for _ in range(200):  # bisection on the monotone P_yy(l2)
        mid = 0.5 * (lo + hi)
        if pyy(mid) > 0:
            hi = mid
        else:
            lo = mid
    l2 = 0.5 * (lo + hi)
    u_aff = np.stack([delta * m.X[:, 0], (l2 - 1) * m.X[:, 1], (l2 - 1) * m.X[:, 2]], 1).reshape(-1)
    assert np.abs(u - u_aff).max() <= 1e-8
    # reaction on x=1: sum of internal forces = P_xx * area(=1)
    R = oracle.residual(m, mat, u)
    nodes = inputs.face_nodes(n, n, n, "x1")
    Pxx = indep.fd_grad(lambda Fm: indep.nh_energy(Fm, E, nu), np.diag([l1, l2, l2]), h=1e-6)[0, 0]
    assert abs(R[3 * nodes].sum() - Pxx) <= 1e-7 * abs(Pxx)


# ------------------------------------------- c0 vs independent assembly ----
def independent_le_solve(w):
    nx, ny, nz = w.nx, w.ny, w.nz
    hx, hy, hz = w.lx / nx, w.ly / ny, w.lz / nz
    Ke = indep.voigt_ke(hx, hy, hz, w.E, w.nu)
    m = oracle.mesh(nx, ny, nz, w.lx, w.ly, w.lz)  # connectivity only
    dofs = (3 * m.conn[:, :, None] + np.arange(3)).reshape(m.n_cells, 24)
    rows = np.repeat(dofs, 24, axis=1).reshape(-1)
    cols = np.tile(dofs, (1, 24)).reshape(-1)
    K = sp.coo_matrix((np.tile(Ke.reshape(-1), m.n_cells), (rows, cols)),
                      shape=(w.n_dofs, w.n_dofs)).tocsr()
    f = indep.face_weight_closed_form(nx, ny, nz, w.lx, w.ly, w.lz, w.traction[0], w.traction[1])
    free = w.mask == 0
    u = np.zeros(w.n_dofs)
    u[free] = spla.spsolve(K[free][:, free].tocsc(), f[free])
    return u


def test_c0_linear_solve_matches_independent_assembly():
    w = inputs.c0()
    m = oracle.mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    mat = oracle.Material(w.kind, w.E, w.nu)
    f = oracle.traction(m, *w.traction)
    u = osolve.linear_solve(m, mat, w.mask, w.u_bar, f)
    ui = independent_le_solve(w)
    assert np.linalg.norm(u - ui) <= 1e-12 * np.linalg.norm(ui)
    R = oracle.residual(m, mat, u, None, f, w.mask)
    assert np.linalg.norm(R) <= 1e-10 * np.linalg.norm(f)
    # the load bends the free end downwards
    assert u[3 * inputs.face_nodes(w.nx, w.ny, w.nz, "x1") + 2].mean() < 0


def test_newton_converges_quadratically():
    w = inputs.c1(n=4, n_steps=2)
    m = oracle.mesh(w.nx, w.ny, w.nz)
    mat = oracle.Material(w.kind, w.E, w.nu)
    hist = []
    osolve.newton_solve(m, mat, w.mask, w.u_bar, n_steps=2, history=hist)
    step1 = [r for s, it, r in hist if s == 1]
    assert len(step1) <= 8
    # quadratic phase: the error ratio drops much faster than linearly
    assert step1[-2] < 1e-3 * step1[0]


# ------------------------------------------------------------ adjoint ------
def small_cantilever(seed=2):
    nx, ny, nz = 4, 2, 2
    mask, ubar = inputs.dirichlet(nx, ny, nz, [("x0", 0, 0.0), ("x0", 1, 0.0), ("x0", 2, 0.0)])
    theta = np.random.default_rng(seed).uniform(0.01, 1.0, nx * ny * nz)
    f = np.zeros(3 * (nx + 1) * (ny + 1) * (nz + 1))
    for node in inputs.face_nodes(nx, ny, nz, "x1")[:4]:
        f[3 * node + 2] = -0.25
    return nx, ny, nz, mask, ubar, theta, f


def test_simp_compliance_gradient_closed_form():
    nx, ny, nz, mask, ubar, theta, f = small_cantilever()
    m = oracle.mesh(nx, ny, nz, 2.0, 1.0, 1.0)
    mat = oracle.Material(oracle.SIMP, 1.0, 0.3, 3.0, 1e-3)
    u = osolve.linear_solve(m, mat, mask, ubar, f, theta)
    g, lam = osolve.adjoint_gradient(m, mat, mask, u, f, theta)
    assert np.linalg.norm(lam - u) <= 1e-10 * np.linalg.norm(u)  # self-adjoint
    K0 = indep.voigt_ke(0.5, 0.5, 0.5, 1.0, 0.3)
    ue = u.reshape(-1, 3)[m.conn].reshape(m.n_cells, 24)
    closed = -3.0 * theta ** 2 * (1 - 1e-3) * np.einsum("ei,ij,ej->e", ue, K0, ue)
    assert np.linalg.norm(g - closed) <= 1e-10 * np.linalg.norm(closed)


def test_simp_compliance_gradient_fd():
    nx, ny, nz, mask, ubar, theta, f = small_cantilever(5)
    m = oracle.mesh(nx, ny, nz, 2.0, 1.0, 1.0)
    mat = oracle.Material(oracle.SIMP, 1.0, 0.3, 3.0, 1e-3)
    pat = osolve._pattern(m)
    u = osolve.linear_solve(m, mat, mask, ubar, f, theta, pat)
    g, _ = osolve.adjoint_gradient(m, mat, mask, u, f, theta, pattern=pat)
    h = 1e-6
    for e in range(0, m.n_cells, 3):
        tp = theta.copy()
        tm = theta.copy()
        tp[e] += h
        tm[e] -= h
        cp = f @ osolve.linear_solve(m, mat, mask, ubar, f, tp, pat)
        cm = f @ osolve.linear_solve(m, mat, mask, ubar, f, tm, pat)
        assert abs(g[e] - (cp - cm) / (2 * h)) <= 1e-6 * np.abs(g).max()


def nh_face_objective_setup(n=3):
    w = inputs.c4(n=n, n_steps=2)
    m = oracle.mesh(n, n, n)
    mat = oracle.Material(oracle.NEOHOOKE, w.E, w.nu)
    nodes = w.extra["face_nodes"]
    target = w.extra["target"]

    def J_of(u):
        d = u.reshape(-1, 3)[nodes] - target
        return np.mean(np.sum(d * d, axis=1))

    def dJdu(u):
        g = np.zeros_like(u).reshape(-1, 3)
        g[nodes] = 2 * (u.reshape(-1, 3)[nodes] - target) / len(nodes)
        return g.reshape(-1)

    return w, m, mat, J_of, dJdu


def test_nh_adjoint_fd_and_taylor():
    w, m, mat, J_of, dJdu = nh_face_objective_setup()
    pat = osolve._pattern(m)

    def Jhat(s):
        u = osolve.newton_solve(m, mat, w.mask, w.u_bar, None, s, n_steps=w.n_steps, pattern=pat)
        return J_of(u), u

    s0 = w.cell_param
    J0, u0 = Jhat(s0)
    g, _ = osolve.adjoint_gradient(m, mat, w.mask, u0, dJdu(u0), s0, pattern=pat)
    # central FD on a few cells
    h = 1e-6
    for e in (0, 13, 26):
        sp_ = s0.copy()
        sm_ = s0.copy()
        sp_[e] += h
        sm_[e] -= h
        fd = (Jhat(sp_)[0] - Jhat(sm_)[0]) / (2 * h)
        assert abs(g[e] - fd) <= 1e-5 * np.abs(g).max()
    # Taylor test, Eqs. (27)-(28): r0 = O(h), r1 = O(h^2)
    ds = np.random.default_rng(17).standard_normal(m.n_cells) * 0.1
    hs = [1e-1, 1e-2, 1e-3, 1e-4]
    r0, r1 = [], []
    for hh in hs:
        Jp = Jhat(s0 + hh * ds)[0]
        r0.append(abs(Jp - J0))
        r1.append(abs(Jp - J0 - hh * g @ ds))
    rate0 = np.polyfit(np.log10(hs), np.log10(r0), 1)[0]
    rate1 = np.polyfit(np.log10(hs[:3]), np.log10(r1[:3]), 1)[0]
    assert 0.9 <= rate0 <= 1.1, r0
    assert 1.8 <= rate1 <= 2.2, r1
