"""The paper's own linear-solve path on the GPU: the tangent assembled by
Algorithm 1 (fem_assemble_csr) and solved by Jacobi-BiCGSTAB
(fem_bicgstab_csr, Sec. 5 item 2), against the oracle's direct solution."""
import numpy as np
import pytest
import torch

import oracle
from oracle import solve as osolve
from paper_2212_00964_gb300 import inputs
from tests.gpu_common import TOL_REFINED, dev, fem, host, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_bicgstab_linear_elastic_c0(prec):
    w = inputs.c0()
    F = fem()
    dt = torch.float64 if prec == "fp64" else torch.float32
    m = F.fem_mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz, csr=True)
    mat = F.material(w.kind, w.E, w.nu)
    vals = F.fem_assemble_csr(m, mat, torch.zeros(w.n_dofs, dtype=dt, device="cuda"), None, dev(w.mask))
    f = torch.zeros(w.n_dofs, dtype=torch.float64, device="cuda")
    F.fem_load_traction(m, w.traction[0], w.traction[1], f)
    b = torch.where(dev(w.mask) != 0, torch.zeros_like(f), f).to(dt)  # prescribed rows: u_bar = 0
    x, it, res = F.fem_bicgstab_csr(m, vals, b, rtol=1e-12 if prec == "fp64" else 1e-6)
    om = oracle.mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    ref = osolve.linear_solve(om, oracle.Material(w.kind, w.E, w.nu), w.mask, w.u_bar,
                              oracle.traction(om, *w.traction))
    assert it > 0 and res <= (1e-12 if prec == "fp64" else 1e-6)
    assert rel_l2(host(x), ref) <= (TOL_REFINED if prec == "fp64" else 1e-4)


def test_bicgstab_neohooke_newton_step():
    """One Newton system K(u) du = -R(u) of the Neo-Hookean box at a random
    state, assembled and solved on the GPU in FP64, against scipy's direct
    solve of the oracle's assembled tangent."""
    n = 6
    w = inputs.c1(n=n, n_steps=1)
    F = fem()
    m = F.fem_mesh(n, n, n, csr=True)
    mat = F.material(w.kind, w.E, w.nu)
    om = oracle.mesh(n, n, n)
    omat = oracle.Material(w.kind, w.E, w.nu)
    u = inputs.random_state(om.n_dofs, 1.0 / n, 5, scale=0.05)
    u[w.mask != 0] = 0.0
    R = F.fem_residual(m, mat, dev(u), None, dev(w.mask))
    vals = F.fem_assemble_csr(m, mat, dev(u), None, dev(w.mask))
    du, it, res = F.fem_bicgstab_csr(m, vals, -R, rtol=1e-12)
    free = w.mask == 0
    Rr = oracle.residual(om, omat, u, None, None, w.mask)
    K = oracle.assemble(om, omat, u)
    ref = np.zeros(om.n_dofs)
    import scipy.sparse.linalg as spla
    ref[free] = spla.spsolve(K[free][:, free].tocsc(), -Rr[free])
    assert res <= 1e-12
    assert rel_l2(host(du), ref) <= TOL_REFINED
