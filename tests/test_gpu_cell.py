"""GPU parity of the cell operators against the oracle, element by element:
residual (Eq. (8) assembled), tangent apply (Eq. (5)), Jacobi diagonal,
adjoint VJP (Eq. (23)), CSR assembly (Algorithm 1).  FP64 within 1e-10 and
FP32 within 1e-5 relative L2, on meshes that span several 128-cell tiles and
end in a ragged tile, with non-cubic boxes and masks."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_00964_gb300 import inputs
from tests.gpu_common import TOL_FP32, TOL_FP64, dev, fem, host, rel_l2

pytestmark = pytest.mark.gpu

MATS = {
    "le": (oracle.LINEAR, 70e3, 0.3),
    "simp": (oracle.SIMP, 1.0, 0.3),
    "nh": (oracle.NEOHOOKE, 10.0, 0.3),
}
SHAPES = [(2, 2, 2), (3, 4, 5), (8, 8, 8), (17, 9, 5)]


def setup(name, shape, seed=0, lengths=(1.0, 0.8, 1.2)):
    kind, E, nu = MATS[name]
    nx, ny, nz = shape
    om = oracle.mesh(nx, ny, nz, *lengths)
    h = min(lengths[0] / nx, lengths[1] / ny, lengths[2] / nz)
    u = inputs.random_state(om.n_dofs, h, seed, scale=0.05)
    x = inputs.random_vector(om.n_dofs, seed + 1)
    rng = np.random.default_rng(seed + 2)
    cp = rng.uniform(0.01, 1.0, om.n_cells) if kind == oracle.SIMP else rng.lognormal(0, 0.5, om.n_cells)
    mask, _ = inputs.clamp_and_compress(nx, ny, nz, -0.1)
    F = fem()
    m = F.fem_mesh(nx, ny, nz, *lengths)
    return F, m, om, oracle.Material(kind, E, nu), F.material(kind, E, nu), u, x, cp, mask


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("name", ["le", "simp", "nh"])
def test_residual_apply_diag_vjp(name, shape, prec):
    F, m, om, omat, gmat, u, x, cp, mask = setup(name, shape)
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = TOL_FP64 if prec == "fp64" else TOL_FP32
    f = inputs.random_vector(om.n_dofs, 99)
    # residual with f_ext and mask
    R_ref = oracle.residual(om, omat, u, cp, f, mask)
    R = F.fem_residual(m, gmat, dev(u, dt), dev(cp, dt), dev(mask), dev(f, dt))
    assert rel_l2(host(R), R_ref) <= tol
    # residual without mask/f_ext
    R0_ref = oracle.residual(om, omat, u, cp)
    assert rel_l2(host(F.fem_residual(m, gmat, dev(u, dt), dev(cp, dt))), R0_ref) <= tol
    # tangent apply with mask
    y_ref = oracle.tangent_apply(om, omat, u, x, cp, mask)
    y = F.fem_tangent_apply(m, gmat, dev(u, dt), dev(x, dt), dev(cp, dt), dev(mask))
    assert rel_l2(host(y), y_ref) <= tol
    y0_ref = oracle.tangent_apply(om, omat, u, x, cp)
    assert rel_l2(host(F.fem_tangent_apply(m, gmat, dev(u, dt), dev(x, dt), dev(cp, dt))), y0_ref) <= tol
    # diagonal
    d_ref = oracle.diag(om, omat, u, cp, mask)
    d = F.fem_tangent_diag(m, gmat, dev(u, dt), dev(cp, dt), dev(mask))
    assert rel_l2(host(d), d_ref) <= tol
    # adjoint VJP
    g_ref = oracle.vjp(om, omat, u, x, cp, mask)
    g = F.fem_vjp(m, gmat, dev(u, dt), dev(x, dt), dev(cp, dt), dev(mask))
    assert rel_l2(host(g), g_ref) <= tol


@pytest.mark.parametrize("name", ["le", "nh"])
def test_no_cell_param_means_unit_scale(name):
    F, m, om, omat, gmat, u, x, cp, mask = setup(name, (3, 4, 5))
    y_ref = oracle.tangent_apply(om, omat, u, x)
    y = F.fem_tangent_apply(m, gmat, dev(u), dev(x))
    assert rel_l2(host(y), y_ref) <= TOL_FP64


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["le", "simp", "nh"])
def test_csr_assembly(name, prec):
    kind, E, nu = MATS[name]
    nx, ny, nz = 3, 4, 5
    om = oracle.mesh(nx, ny, nz, 1.0, 0.8, 1.2)
    u = inputs.random_state(om.n_dofs, 0.2, 4, scale=0.05)
    rng = np.random.default_rng(5)
    cp = rng.uniform(0.01, 1.0, om.n_cells) if kind == oracle.SIMP else rng.lognormal(0, 0.5, om.n_cells)
    mask, _ = inputs.clamp_and_compress(nx, ny, nz, -0.1)
    F = fem()
    m = F.fem_mesh(nx, ny, nz, 1.0, 0.8, 1.2, csr=True)
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = TOL_FP64 if prec == "fp64" else TOL_FP32
    rp, col = oracle.csr(om)
    smap = oracle.scatter_map(om, rp, col)
    omat = oracle.Material(kind, E, nu)
    for mk in (None, mask):
        ref = oracle.assemble_vals(om, omat, u, rp, col, smap, cp, mk)
        got = F.fem_assemble_csr(m, F.material(kind, E, nu), dev(u, dt), dev(cp, dt),
                                 None if mk is None else dev(mk))
        assert rel_l2(host(got), ref) <= tol


def test_loads_match_oracle():
    F = fem()
    nx, ny, nz, L = 5, 3, 4, (1.0, 0.5, 2.0)
    m = F.fem_mesh(nx, ny, nz, *L)
    om = oracle.mesh(nx, ny, nz, *L)
    f = torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda")
    for face in ("x0", "x1", "y0", "y1", "z0", "z1"):
        t = (0.3, -1.0, 2.0)
        f.zero_()
        F.fem_load_traction(m, face, t, f)
        assert rel_l2(host(f), oracle.traction(om, face, t)) <= 1e-14
    f.zero_()
    F.fem_load_body(m, (1.0, 2.0, -3.0), f)
    b = np.tile([1.0, 2.0, -3.0], (om.n_cells, 8, 1))
    assert rel_l2(host(f), oracle.body_force(om, b)) <= 1e-14


@pytest.mark.parametrize("case", ["c1_nh_64cube", "c2_simp_128x64x64", "c2_simp_128x64x64_tensor_cores"])
def test_full_size_apply_sampled(case):
    """FP32 tangent apply in the benchmark configurations (the 64^3
    Neo-Hookean box on the packed CUDA-core kernel, the 128x64x64 SIMP
    cantilever on the CUDA cores and on the tensor cores; many cell tiles per
    CTA): sampled
    output DOFs against the oracle apply restricted to the cells around each
    sampled node (computed one by one on a sub-box)."""
    F = fem()
    w = inputs.c1(64) if case.startswith("c1") else inputs.c2()
    nx, ny, nz = w.nx, w.ny, w.nz
    hx, hy, hz = w.lx / nx, w.ly / ny, w.lz / nz
    m = F.fem_mesh(nx, ny, nz, w.lx, w.ly, w.lz, tensor_cores=case.endswith("tensor_cores"))
    u = inputs.random_state(w.n_dofs, min(hx, hy, hz), 11, scale=0.05)
    x = inputs.random_vector(w.n_dofs, 12)
    cp = w.cell_param
    gmat = F.material(w.kind, w.E, w.nu, w.simp_p, w.simp_emin)
    y = host(F.fem_tangent_apply(m, gmat, dev(u, torch.float32), dev(x, torch.float32),
                                 None if cp is None else dev(cp, torch.float32), dev(w.mask)))
    omat = oracle.Material(w.kind, w.E, w.nu, w.simp_p, w.simp_emin)
    ax, ay = nx + 1, ny + 1
    rng = np.random.default_rng(3)
    for node in rng.integers(0, w.n_nodes, 12):
        I, J, K = node % ax, (node // ax) % ay, node // (ax * ay)
        i0, j0, k0 = max(I - 1, 0), max(J - 1, 0), max(K - 1, 0)
        i1, j1, k1 = min(I + 1, nx), min(J + 1, ny), min(K + 1, nz)
        sub = oracle.mesh(i1 - i0, j1 - j0, k1 - k0, (i1 - i0) * hx, (j1 - j0) * hy, (k1 - k0) * hz)
        II, JJ, KK = np.meshgrid(np.arange(i0, i1 + 1), np.arange(j0, j1 + 1), np.arange(k0, k1 + 1), indexing="ij")
        gid = (II + ax * (JJ + ay * KK)).transpose(2, 1, 0).reshape(-1)  # sub-node order x fastest
        dofs = (3 * gid[:, None] + np.arange(3)).reshape(-1)
        sub_cp = None
        if cp is not None:
            CI, CJ, CK = np.meshgrid(np.arange(i0, i1), np.arange(j0, j1), np.arange(k0, k1), indexing="ij")
            sub_cp = cp[(CI + nx * (CJ + ny * CK)).transpose(2, 1, 0).reshape(-1)]
        ys = oracle.tangent_apply(sub, omat, u[dofs], x[dofs], sub_cp, w.mask[dofs])
        loc = int(np.where(gid == node)[0][0])
        ref = ys[3 * loc:3 * loc + 3]
        got = y[3 * node:3 * node + 3]
        assert np.abs(got - ref).max() <= 3e-5 * np.abs(ys).max(), (node, got, ref)


@pytest.mark.parametrize("name", ["le", "simp"])
def test_tensor_core_apply_as_accurate_as_fp32(name):
    """On a FEM_MESH_TENSOR_CORES mesh the FP32 linear-elastic / SIMP apply
    runs on the tensor cores (split-TF32 products of the shared element
    matrix); it matches the oracle like the other FP32 applies (ragged tiles,
    masks) and its error against the FP64 apply stays within three times
    that of the FP32 CUDA-core kernel on the same inputs, and within 1e-6
    relative L2."""
    F, _, om, omat, gmat, u, x, cp, mask = setup(name, (17, 9, 5))
    mt = F.fem_mesh(17, 9, 5, 1.0, 0.8, 1.2, tensor_cores=True)
    f32 = torch.float32
    for mk in (mask, None):
        y_ref = oracle.tangent_apply(om, omat, u, x, cp, mk)
        y = F.fem_tangent_apply(mt, gmat, dev(u, f32), dev(x, f32), dev(cp, f32), None if mk is None else dev(mk))
        assert rel_l2(host(y), y_ref) <= TOL_FP32
    shape = (64, 32, 16)
    F, m, om, omat, gmat, u, x, cp, mask = setup(name, shape)
    mt = F.fem_mesh(*shape, 1.0, 0.8, 1.2, tensor_cores=True)
    y64 = host(F.fem_tangent_apply(m, gmat, dev(u), dev(x), dev(cp), dev(mask)))
    y_tc = host(F.fem_tangent_apply(mt, gmat, dev(u, f32), dev(x, f32), dev(cp, f32), dev(mask)))
    y_cc = host(F.fem_tangent_apply(m, gmat, dev(u, f32), dev(x, f32), dev(cp, f32), dev(mask)))
    e_tc, e_cc = rel_l2(y_tc, y64), rel_l2(y_cc, y64)
    assert e_tc <= 1e-6 and e_tc <= 3.0 * e_cc, (e_tc, e_cc)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 4, 5), (17, 9, 5)])
def test_deterministic_mesh_colour_ordered(shape, prec):
    """FEM_MESH_DETERMINISTIC: the cell operators scatter colour by colour
    (a2) with plain stores.  Same parity bar as the atomic path, and two runs
    agree bit for bit (1x1x1 has a single non-empty colour class)."""
    F, _, om, omat, gmat, u, x, cp, mask = setup("nh", shape)
    nx, ny, nz = shape
    md = F.fem_mesh(nx, ny, nz, 1.0, 0.8, 1.2, deterministic=True)
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = TOL_FP64 if prec == "fp64" else TOL_FP32
    f = inputs.random_vector(om.n_dofs, 99)
    R_ref = oracle.residual(om, omat, u, cp, f, mask)
    y_ref = oracle.tangent_apply(om, omat, u, x, cp, mask)
    d_ref = oracle.diag(om, omat, u, cp, mask)
    runs = []
    for _ in range(2):
        R = F.fem_residual(md, gmat, dev(u, dt), dev(cp, dt), dev(mask), dev(f, dt))
        y = F.fem_tangent_apply(md, gmat, dev(u, dt), dev(x, dt), dev(cp, dt), dev(mask))
        d = F.fem_tangent_diag(md, gmat, dev(u, dt), dev(cp, dt), dev(mask))
        runs.append((host(R), host(y), host(d)))
    for got, ref in zip(runs[0], (R_ref, y_ref, d_ref)):
        assert rel_l2(got, ref) <= tol
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(a, b)
