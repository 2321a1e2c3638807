"""Pins of the oracle's global operators: residual (Eq. (2) discretised),
matrix-free tangent (Eq. (5)), diagonal, assembly (Algorithm 1), adjoint VJP
(Eq. (23)), external loads."""
import numpy as np
import pytest

import oracle
from paper_2212_00964_gb300 import inputs
from tests import indep

MATS = {
    "le": oracle.Material(oracle.LINEAR, 70e3, 0.3),
    "simp": oracle.Material(oracle.SIMP, 1.0, 0.3, 3.0, 1e-3),
    "nh": oracle.Material(oracle.NEOHOOKE, 10.0, 0.3),
}


def perturbed(m, amp, seed):
    rng = np.random.default_rng(seed)
    h = min(m.lx / m.nx, m.ly / m.ny, m.lz / m.nz)
    X = m.X + amp * h * rng.uniform(-1, 1, m.X.shape)
    return oracle.with_coords(m, X)


def interior_dofs(m):
    n = np.arange(m.n_nodes)
    i = n % (m.nx + 1)
    j = (n // (m.nx + 1)) % (m.ny + 1)
    k = n // ((m.nx + 1) * (m.ny + 1))
    inner = (i > 0) & (i < m.nx) & (j > 0) & (j < m.ny) & (k > 0) & (k < m.nz)
    return np.repeat(inner, 3)


def cell_param_for(kind, ne, seed):
    rng = np.random.default_rng(seed)
    if kind == oracle.SIMP:
        return rng.uniform(0.01, 1.0, ne)
    return rng.lognormal(0, 0.5, ne)


@pytest.mark.parametrize("name", ["le", "simp", "nh"])
def test_patch_test_affine_field(name):
    """An affine displacement u = A X + b has constant grad u, so every
    interior node's residual vanishes on any (perturbed) mesh."""
    mat = MATS[name]
    m = perturbed(oracle.mesh(4, 3, 5, 1.0, 0.8, 1.2), 0.2, 42)
    rng = np.random.default_rng(7)
    A = 0.05 * rng.standard_normal((3, 3))
    u = (m.X @ A.T + rng.standard_normal(3) * 0.01).reshape(-1)
    cp = np.full(m.n_cells, 0.6) if mat.kind == oracle.SIMP else None
    R = oracle.residual(m, mat, u, cp)
    inner = interior_dofs(m)
    scale = np.abs(R[~inner]).max()
    assert scale > 0
    assert np.abs(R[inner]).max() <= 1e-12 * scale


@pytest.mark.parametrize("name", ["le", "simp", "nh"])
def test_tangent_is_residual_derivative(name):
    """JVP = central FD of the residual on a 2x2x2 mesh."""
    mat = MATS[name]
    m = perturbed(oracle.mesh(2, 2, 2), 0.15, 3)
    u = inputs.random_state(m.n_dofs, 0.5, 5, scale=0.1)
    x = inputs.random_vector(m.n_dofs, 6)
    cp = cell_param_for(mat.kind, m.n_cells, 9)
    y = oracle.tangent_apply(m, mat, u, x, cp)
    h = 1e-6
    fd = (oracle.residual(m, mat, u + h * x, cp) - oracle.residual(m, mat, u - h * x, cp)) / (2 * h)
    assert np.linalg.norm(y - fd) <= 1e-7 * np.linalg.norm(y)


@pytest.mark.parametrize("name", ["le", "simp", "nh"])
def test_tangent_symmetric(name):
    mat = MATS[name]
    m = perturbed(oracle.mesh(3, 2, 2), 0.1, 4)
    u = inputs.random_state(m.n_dofs, 0.4, 8, scale=0.1)
    v = inputs.random_vector(m.n_dofs, 1)
    w = inputs.random_vector(m.n_dofs, 2)
    cp = cell_param_for(mat.kind, m.n_cells, 10)
    mask, _ = inputs.dirichlet(3, 2, 2, [("x0", 0, 0.0), ("x0", 1, 0.0), ("y1", 2, 0.0)])
    Kv = oracle.tangent_apply(m, mat, u, v, cp, mask)
    Kw = oracle.tangent_apply(m, mat, u, w, cp, mask)
    assert abs(w @ Kv - v @ Kw) <= 1e-12 * np.linalg.norm(Kv) * np.linalg.norm(w)


def test_nh_global_tangent_at_zero_is_le():
    m = perturbed(oracle.mesh(3, 3, 2), 0.1, 12)
    E, nu = 10.0, 0.3
    x = inputs.random_vector(m.n_dofs, 4)
    a = oracle.tangent_apply(m, oracle.Material(oracle.NEOHOOKE, E, nu), np.zeros(m.n_dofs), x)
    b = oracle.tangent_apply(m, oracle.Material(oracle.LINEAR, E, nu), np.zeros(m.n_dofs), x)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_le_residual_is_linear():
    mat = MATS["le"]
    m = perturbed(oracle.mesh(2, 3, 2), 0.1, 2)
    u = inputs.random_vector(m.n_dofs, 3)
    R = oracle.residual(m, mat, u)
    y = oracle.tangent_apply(m, mat, np.zeros(m.n_dofs), u)
    assert np.linalg.norm(R - y) <= 1e-12 * np.linalg.norm(y)


@pytest.mark.parametrize("name", ["le", "simp", "nh"])
def test_mask_semantics_diag_and_assembly(name):
    mat = MATS[name]
    nx, ny, nz = 3, 2, 2
    m = oracle.mesh(nx, ny, nz)
    u = inputs.random_state(m.n_dofs, 1 / 3, 21, scale=0.1)
    x = inputs.random_vector(m.n_dofs, 22)
    cp = cell_param_for(mat.kind, m.n_cells, 23)
    mask, _ = inputs.clamp_and_compress(nx, ny, nz, -0.1)
    c = mask.astype(bool)
    f = inputs.random_vector(m.n_dofs, 24)
    R = oracle.residual(m, mat, u, cp, f, mask)
    R0 = oracle.residual(m, mat, u, cp)
    assert np.all(R[c] == 0) and np.allclose(R[~c], R0[~c] - f[~c], rtol=0, atol=1e-12 * np.abs(R0).max())
    y = oracle.tangent_apply(m, mat, u, x, cp, mask)
    assert np.all(y[c] == x[c])
    xm = np.where(c, 0.0, x)
    y0 = oracle.tangent_apply(m, mat, u, xm, cp)
    assert np.allclose(y[~c], y0[~c], rtol=0, atol=1e-12 * np.abs(y0).max())
    K = oracle.assemble(m, mat, u, cp, mask).toarray()
    assert np.allclose(K @ x, y, rtol=0, atol=1e-11 * np.abs(y).max())
    d = oracle.diag(m, mat, u, cp, mask)
    assert np.allclose(np.diag(K), d, rtol=0, atol=1e-12 * np.abs(d).max())
    Kfull = oracle.assemble(m, mat, u, cp).toarray()
    # column by column: K e_j = JVP with unit vector
    for j in [0, 7, 31, m.n_dofs - 1]:
        ej = np.zeros(m.n_dofs)
        ej[j] = 1
        assert np.allclose(Kfull[:, j], oracle.tangent_apply(m, mat, u, ej, cp), atol=1e-12 * np.abs(Kfull).max())


@pytest.mark.parametrize("name", ["simp", "nh", "le"])
def test_vjp_is_parameter_derivative(name):
    """g_e = -lambda^T dR/dtheta_e, checked by central FD in theta_e."""
    mat = MATS[name]
    nx, ny, nz = 3, 2, 2
    m = oracle.mesh(nx, ny, nz)
    u = inputs.random_state(m.n_dofs, 0.5, 31, scale=0.1)
    lam = inputs.random_vector(m.n_dofs, 32)
    cp = cell_param_for(mat.kind, m.n_cells, 33)
    mask, _ = inputs.clamp_and_compress(nx, ny, nz, -0.1)
    g = oracle.vjp(m, mat, u, lam, cp, mask)
    lamm = np.where(mask.astype(bool), 0.0, lam)
    h = 1e-6
    for e in range(m.n_cells):
        cpp = cp.copy()
        cpm = cp.copy()
        cpp[e] += h
        cpm[e] -= h
        fd = -(lamm @ (oracle.residual(m, mat, u, cpp, None, mask) - oracle.residual(m, mat, u, cpm, None, mask))) / (2 * h)
        assert abs(g[e] - fd) <= 1e-7 * max(1.0, np.abs(g).max())


@pytest.mark.parametrize("face", ["x0", "x1", "y0", "y1", "z0", "z1"])
def test_traction_closed_form(face):
    nx, ny, nz, lx, ly, lz = 3, 4, 2, 1.0, 2.0, 0.5
    m = oracle.mesh(nx, ny, nz, lx, ly, lz)
    t = (1.5, -2.0, 0.25)
    f = oracle.traction(m, face, t)
    fc = indep.face_weight_closed_form(nx, ny, nz, lx, ly, lz, face, t)
    assert np.abs(f - fc).max() <= 1e-13 * np.abs(fc).max()


def test_traction_total_force_on_perturbed_interior():
    m = oracle.mesh(4, 4, 4)
    t = (0.0, 0.0, -100.0)
    f = oracle.traction(m, "x1", t)
    assert np.allclose(f.reshape(-1, 3).sum(0), t, atol=1e-12)
