"""GPU adjoint gradient (Sec. 3, Eqs. (22)-(23)) against the oracle adjoint
(<= 1e-6), central finite differences (<= 1e-4) and, for compliance, the
self-adjoint closed form; plus the torch.autograd.Function around it."""
import numpy as np
import pytest
import torch

import oracle
from oracle import solve as osolve
from paper_2212_00964_gb300 import inputs
from tests.gpu_common import TOL_ADJ_FD, TOL_ADJ_ORACLE, TOL_REFINED, dev, fem, host, rel_l2

pytestmark = pytest.mark.gpu


def simp_problem(nx=16, ny=8, nz=8):
    w = inputs.c2(nx=nx, ny=ny, nz=nz)
    return w


def gpu_forward(F, m, w, theta, precision=2, **opt):
    u = torch.zeros(w.n_dofs, dtype=torch.float64, device="cuda")
    f = dev(w.point_load) if w.point_load is not None else None
    o = F.default_options(precision=precision, **opt)
    F.fem_solve(m, F.material(w.kind, w.E, w.nu, w.simp_p, w.simp_emin), dev(w.mask), dev(w.u_bar), u, f,
                dev(theta), w.n_steps, o)
    return u


def test_simp_compliance_adjoint_vs_oracle_and_fd():
    F = fem()
    w = simp_problem()
    m = F.fem_mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    mat = F.material(w.kind, w.E, w.nu, w.simp_p, w.simp_emin)
    theta = w.cell_param
    u = gpu_forward(F, m, w, theta, newton_rtol=1e-12)
    f = dev(w.point_load)
    g, st = F.fem_adjoint(m, mat, dev(w.mask), u, f, dev(theta), options=F.default_options(newton_rtol=1e-12))
    assert st["status"] == 0
    om = oracle.mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    omat = oracle.Material(w.kind, w.E, w.nu, w.simp_p, w.simp_emin)
    u_ref = osolve.linear_solve(om, omat, w.mask, w.u_bar, w.point_load, theta)
    g_ref, _ = osolve.adjoint_gradient(om, omat, w.mask, u_ref, w.point_load, theta)
    assert rel_l2(host(g), g_ref) <= TOL_ADJ_ORACLE
    # central FD of the compliance C = f.u on a few cells (FP64 GPU solves)
    h = 1e-5
    for e in inputs.fd_cells(om.n_cells, k=6):
        tp = theta.copy()
        tm = theta.copy()
        tp[e] += h
        tm[e] -= h
        cp_ = float(f @ gpu_forward(F, m, w, tp, 0, newton_rtol=1e-12, pcg_rtol=1e-10))
        cm_ = float(f @ gpu_forward(F, m, w, tm, 0, newton_rtol=1e-12, pcg_rtol=1e-10))
        fd = (cp_ - cm_) / (2 * h)
        assert abs(float(g[e]) - fd) <= TOL_ADJ_FD * np.abs(g_ref).max()


def face_objective(w):
    nodes = torch.as_tensor(w.extra["face_nodes"], device="cuda")
    target = torch.as_tensor(w.extra["target"], device="cuda")

    def J(u):
        d = u.view(-1, 3)[nodes] - target
        return (d * d).sum(dim=1).mean()

    return J


def test_neohooke_face_objective_adjoint_vs_oracle_and_fd():
    F = fem()
    n = 4
    w = inputs.c4(n=n, n_steps=2)
    m = F.fem_mesh(n, n, n)
    mat = F.material(w.kind, w.E, w.nu)
    s = w.cell_param
    J = face_objective(w)
    u = gpu_forward(F, m, w, s, newton_rtol=1e-12)
    uu = u.clone().requires_grad_(True)
    dJdu = torch.autograd.grad(J(uu), uu)[0].contiguous()
    g, st = F.fem_adjoint(m, mat, dev(w.mask), u, dJdu, dev(s), options=F.default_options(newton_rtol=1e-12))
    om = oracle.mesh(n, n, n)
    omat = oracle.Material(w.kind, w.E, w.nu)
    u_ref = osolve.newton_solve(om, omat, w.mask, w.u_bar, None, s, n_steps=2)
    g_ref, _ = osolve.adjoint_gradient(om, omat, w.mask, u_ref, host(dJdu), s)
    assert rel_l2(host(g), g_ref) <= TOL_ADJ_ORACLE
    h = 1e-5
    for e in (0, 21, 63):
        sp_ = s.copy()
        sm_ = s.copy()
        sp_[e] += h
        sm_[e] -= h
        jp = float(J(gpu_forward(F, m, w, sp_, 0, newton_rtol=1e-12, pcg_rtol=1e-10)))
        jm = float(J(gpu_forward(F, m, w, sm_, 0, newton_rtol=1e-12, pcg_rtol=1e-10)))
        assert abs(float(g[e]) - (jp - jm) / (2 * h)) <= TOL_ADJ_FD * np.abs(g_ref).max()


def test_autograd_function_matches_adjoint():
    from paper_2212_00964_gb300.autograd import FemSolve
    F = fem()
    n = 4
    w = inputs.c4(n=n, n_steps=2)
    m = F.fem_mesh(n, n, n)
    solver = FemSolve(m, F.material(w.kind, w.E, w.nu), dev(w.mask), dev(w.u_bar), n_steps=2,
                      options=F.default_options(newton_rtol=1e-12))
    theta = dev(w.cell_param).requires_grad_(True)
    J = face_objective(w)
    loss = J(solver(theta))
    (g,) = torch.autograd.grad(loss, theta)
    om = oracle.mesh(n, n, n)
    omat = oracle.Material(w.kind, w.E, w.nu)
    u_ref = osolve.newton_solve(om, omat, w.mask, w.u_bar, None, w.cell_param, n_steps=2)
    nodes = w.extra["face_nodes"]
    dJ = np.zeros_like(u_ref).reshape(-1, 3)
    dJ[nodes] = 2 * (u_ref.reshape(-1, 3)[nodes] - w.extra["target"]) / len(nodes)
    g_ref, _ = osolve.adjoint_gradient(om, omat, w.mask, u_ref, dJ.reshape(-1), w.cell_param)
    assert rel_l2(host(g), g_ref) <= TOL_ADJ_ORACLE


@pytest.mark.slow
def test_c2_full_size_compliance_closed_form():
    """128x64x64 SIMP cantilever: the GPU adjoint gradient of the compliance
    equals the self-adjoint closed form -s'(theta_e) u_e^T K0_e u_e at the
    GPU solution (oracle VJP with lambda = u), and central FD of the
    compliance on the 64 cells drawn with seed 7, each side a full-size
    mixed-precision solve."""
    F = fem()
    w = inputs.c2()
    m = F.fem_mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    mat = F.material(w.kind, w.E, w.nu, w.simp_p, w.simp_emin)
    u = gpu_forward(F, m, w, w.cell_param, newton_rtol=1e-11)
    f = dev(w.point_load)
    g, st = F.fem_adjoint(m, mat, dev(w.mask), u, f, dev(w.cell_param))
    assert st["status"] == 0
    om = oracle.mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    omat = oracle.Material(w.kind, w.E, w.nu, w.simp_p, w.simp_emin)
    closed = oracle.vjp(om, omat, host(u), host(u), w.cell_param, w.mask)
    assert rel_l2(host(g), closed) <= TOL_ADJ_ORACLE
    h = 1e-4
    cells = inputs.fd_cells(om.n_cells, k=64, seed=7)
    assert cells.size == 64
    for e in cells:
        tp = w.cell_param.copy()
        tm = w.cell_param.copy()
        tp[e] += h
        tm[e] -= h
        cp_ = float(f @ gpu_forward(F, m, w, tp, 2, newton_rtol=1e-12))
        cm_ = float(f @ gpu_forward(F, m, w, tm, 2, newton_rtol=1e-12))
        assert abs(float(g[e]) - (cp_ - cm_) / (2 * h)) <= TOL_ADJ_FD * np.abs(closed).max()


@pytest.mark.slow
def test_c4_full_size_forward_and_adjoint_properties():
    """128^3 Neo-Hookean with a log-normal stiffness field, 5 load steps, at
    full size (6.4M DOF, beyond the oracle's direct solver), by properties
    that hold at any size: the oracle's FP64 residual at the mixed-precision
    GPU solution is at the Newton tolerance; the GPU adjoint variable solves
    the oracle's tangent system K(u) lambda = dJ/du on the free DOFs; and the
    GPU gradient equals the oracle's vector-Jacobian product at that lambda;
    and the mixed-precision solution equals the all-FP64 GPU solution to
    relative L2 1e-8."""
    F = fem()
    w = inputs.c4()
    m = F.fem_mesh(w.nx, w.ny, w.nz)
    mat = F.material(w.kind, w.E, w.nu)
    J = face_objective(w)
    o = F.default_options(newton_rtol=1e-10)
    u = torch.zeros(w.n_dofs, dtype=torch.float64, device="cuda")
    st = F.fem_solve(m, mat, dev(w.mask), dev(w.u_bar), u, None, dev(w.cell_param), w.n_steps, o)
    assert st["status"] == 0 and st["load_steps"] == w.n_steps
    om = oracle.mesh(w.nx, w.ny, w.nz)
    omat = oracle.Material(w.kind, w.E, w.nu)
    uh = host(u)
    R = oracle.residual(om, omat, uh, w.cell_param, None, w.mask)
    assert np.linalg.norm(R) <= 1e-9 * st["ref_rnorm"]
    uu = u.clone().requires_grad_(True)
    dJdu = torch.autograd.grad(J(uu), uu)[0].contiguous()
    lam = torch.zeros_like(u)
    g, sta = F.fem_adjoint(m, mat, dev(w.mask), u, dJdu, dev(w.cell_param), options=o, lam=lam)
    assert sta["status"] == 0
    lh, b = host(lam), host(dJdu)
    free = w.mask == 0
    assert np.all(lh[~free] == 0)
    Kl = oracle.tangent_apply(om, omat, uh, lh, w.cell_param, w.mask)
    assert np.linalg.norm((Kl - b)[free]) <= 1e-8 * np.linalg.norm(b[free])
    g_ref = oracle.vjp(om, omat, uh, lh, w.cell_param, w.mask)
    assert rel_l2(host(g), g_ref) <= TOL_ADJ_ORACLE
    u64 = torch.zeros_like(u)
    o64 = F.default_options(precision=F.FEM_FP64, newton_rtol=1e-10)
    st64 = F.fem_solve(m, mat, dev(w.mask), dev(w.u_bar), u64, None, dev(w.cell_param), w.n_steps, o64)
    assert st64["status"] == 0
    assert rel_l2(uh, host(u64)) <= TOL_REFINED
