"""GPU parity of the topology-optimisation steps (Sec. 3.2): the cone filter
(fem_density_filter) and the MMA step (fem_mma_step) against the oracle,
and the whole design loop on the box cantilever with the GPU's SIMP solve
and compliance gradient (fem_solve, fem_adjoint)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import topopt as ot
from paper_2212_00964_gb300 import inputs
from tests.gpu_common import dev, fem, host, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rmin", [1.0, 1.5, 2.3])
def test_filter_parity(rmin):
    nx, ny, nz = 37, 9, 5
    F = fem()
    m = F.fem_mesh(nx, ny, nz)
    g = np.random.default_rng(4).standard_normal(nx * ny * nz)
    out = F.fem_density_filter(m, dev(g), rmin)
    ref = ot.filter_sensitivities(ot.filter_matrix(nx, ny, nz, rmin), g)
    assert rel_l2(host(out), ref) <= 1e-14


@pytest.mark.parametrize("rmin", [1.5, 2.3])
def test_filter_transpose_parity(rmin):
    nx, ny, nz = 21, 8, 5
    F = fem()
    m = F.fem_mesh(nx, ny, nz)
    g = np.random.default_rng(6).standard_normal(nx * ny * nz)
    out = F.fem_density_filter(m, dev(g), rmin, transpose=True)
    ref = ot.filter_transpose(ot.filter_matrix(nx, ny, nz, rmin), g)
    assert rel_l2(host(out), ref) <= 1e-14


def test_oc_steps_parity():
    F = fem()
    m = F.fem_mesh(6, 5, 4)
    n = m.n_cells
    rng = np.random.default_rng(7)
    c = rng.uniform(0.2, 1.0, n)
    dv = rng.uniform(0.5, 1.5, n)
    x = np.full(n, 0.4)
    for it in range(8):
        g = -c / x ** 2
        ref, lam_ref = ot.oc_step(x, g, dv, 0.4, 0.15, 0.01, 1.0)
        y, lam = F.fem_oc_step(m, dev(x), dev(g), dev(dv), 0.4, 0.15, 0.01, 1.0)
        assert abs(lam - lam_ref) <= 1e-12 * lam_ref
        assert np.abs(host(y) - ref).max() <= 1e-12, it
        x = ref


def test_mma_steps_parity():
    """Twelve steps on min sum c/x under a mean constraint, oracle and GPU
    fed the same iterates."""
    F = fem()
    m = F.fem_mesh(6, 5, 4)
    n = m.n_cells
    rng = np.random.default_rng(5)
    c = rng.uniform(0.2, 1.0, n)
    ref = ot.MMA(n, 0.01, 1.0)
    st = F.MMAState(m, 0.01, 1.0)
    x = np.full(n, 0.4)
    for it in range(12):
        args = (np.sum(c / x), -c / x ** 2, x.mean() - 0.4, np.full(n, 1.0 / n))
        y_ref = ref.step(x, *args)
        y = st.step(dev(x), args[2], dev(args[1]), dev(args[3]))
        assert np.abs(host(y) - y_ref).max() <= 1e-12, it
        x = y_ref


def test_design_loop_on_box_cantilever():
    """The loop with every data-parallel step on the GPU: after 40
    iterations the volume constraint is active and the compliance is within
    1% of the oracle loop's."""
    w = inputs.topopt_cantilever()
    F = fem()
    m = F.fem_mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    mat = F.material(w.kind, w.E, w.nu, w.simp_p, w.simp_emin)
    om = oracle.mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    omat = oracle.Material(oracle.SIMP, w.E, w.nu, w.simp_p, w.simp_emin)
    hist = []
    th_ref = ot.optimise(om, omat, w.mask, w.point_load, 0.5, 1.5, 40, history=hist)
    c_ref = ot.compliance_and_gradient(om, omat, w.mask, w.point_load, th_ref)[0]
    mask, f = dev(w.mask), dev(w.point_load)
    zero = torch.zeros(om.n_dofs, dtype=torch.float64, device="cuda")
    theta = torch.full((om.n_cells,), 0.5, dtype=torch.float64, device="cuda")
    st = F.MMAState(m, 0.0, 1.0)
    dv = torch.full_like(theta, 1.0 / om.n_cells)
    opts = F.default_options(precision=F.FEM_FP64, newton_rtol=1e-12)
    cs = []
    for it in range(40):
        u = torch.zeros_like(zero)
        F.fem_solve(m, mat, mask, zero, u, f, theta, options=opts)
        cs.append(float(f @ u))
        g, _ = F.fem_adjoint(m, mat, mask, u, f, theta, options=opts)
        gf = F.fem_density_filter(m, g, 1.5)
        theta = st.step(theta, float(theta.mean()) - 0.5, gf, dv)
    assert abs(cs[0] - hist[0][0]) <= 1e-8 * cs[0]
    assert abs(float(theta.mean()) - 0.5) <= 1e-4
    u = torch.zeros_like(zero)
    F.fem_solve(m, mat, mask, zero, u, f, theta, options=opts)
    assert abs(float(f @ u) - c_ref) <= 0.01 * c_ref


def test_hyperelastic_simp_steps():
    """The paper's plate physics: SIMP on the Neo-Hookean law through the
    main path (per-cell stiffness scale s(theta), fem_solve + fem_adjoint in
    FP64) with the chain rule ds/dtheta, then filter and MMA step, against
    the oracle on the same designs for six iterations."""
    w = inputs.topopt_cantilever(nx=8, ny=4, nz=4, lx=2.0, ly=1.0, lz=1.0)
    F = fem()
    m = F.fem_mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    om = oracle.mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    f_h = w.point_load * 2e-3
    mat = F.material(F.FEM_NEOHOOKE, 1.0, 0.3)
    opts = F.default_options(precision=F.FEM_FP64, newton_rtol=1e-12)
    mask, f = dev(w.mask), dev(f_h)
    zero = torch.zeros(om.n_dofs, dtype=torch.float64, device="cuda")
    H = ot.filter_matrix(w.nx, w.ny, w.nz, 1.5)
    ref_mma = ot.MMA(om.n_cells, 0.0, 1.0)
    st = F.MMAState(m, 0.0, 1.0)
    dv = np.full(om.n_cells, 1.0 / om.n_cells)
    theta = np.full(om.n_cells, 0.5)
    for it in range(6):
        c_ref, g_ref, _ = ot.compliance_and_gradient_nh(om, 1.0, 0.3, w.mask, f_h, theta)
        th = dev(theta)
        s = 1e-3 + th ** 3 * (1 - 1e-3)
        u = torch.zeros_like(zero)
        F.fem_solve(m, mat, mask, zero, u, f, s, options=opts)
        g_s, _ = F.fem_adjoint(m, mat, mask, u, f, s, options=opts)
        g = g_s * 3 * th ** 2 * (1 - 1e-3)
        c = float(f @ u)
        assert abs(c - c_ref) <= 1e-8 * c_ref, it
        assert rel_l2(host(g), g_ref) <= 1e-6, it
        gf = F.fem_density_filter(m, g, 1.5)
        y = st.step(th, float(theta.mean()) - 0.5, gf, dev(dv))
        y_ref = ref_mma.step(theta, c_ref, ot.filter_sensitivities(H, g_ref), float(theta.mean() - 0.5), dv)
        assert np.abs(host(y) - y_ref).max() <= 1e-6, it
        theta = y_ref


def test_mma_infeasible_constraint_is_not_converged():
    F = fem()
    m = F.fem_mesh(2, 1, 1)
    st = F.MMAState(m, 0.0, 1.0)
    x = dev(np.array([0.5, 0.7]))
    with pytest.raises(F.FemError) as e:
        st.step(x, 2.0 - 0.6, dev(np.zeros(2)), dev(np.full(2, -0.5)))
    assert e.value.status == F.FEM_ERR_NOT_CONVERGED
