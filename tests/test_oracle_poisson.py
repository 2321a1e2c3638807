"""Pins of the scalar Poisson oracle (Sec. 3.1, Eqs. (24)-(28)): element
matrices against their tensor-product closed forms, the patch test, a
manufactured solution, the adjoint gradient against exact central
differences and the Taylor remainders of Eqs. (27)-(28), and the paper's
printed inference errors."""
import os

import numpy as np
import pytest

import oracle
from oracle import poisson as op
from paper_2212_00964_gb300 import inputs
from tests import indep

K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])          # int_0^1 phi_i' phi_j' (unit interval)
M1 = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])    # int_0^1 phi_i phi_j


def corner_bits(m, e=0):
    """0/1 position of each local node of cell e along x, y, z (from the
    node coordinates, not from the oracle's corner table)."""
    X = m.X[m.conn[e]]
    lo, hi = X.min(axis=0), X.max(axis=0)
    return np.rint((X - lo) / (hi - lo)).astype(int)


def tensor_product_matrices(bits, h, alpha):
    """Ke, Me of an axis-aligned box cell as sums of Kronecker-type products
    of the 1D linear-element matrices: K_ab = alpha V sum_d h_d^-2 K1 x M1 x M1
    (K1 on axis d), M_ab = V M1 x M1 x M1."""
    V = np.prod(h)
    Ke = np.zeros((8, 8))
    Me = np.zeros((8, 8))
    for a in range(8):
        for b in range(8):
            m1 = [M1[bits[a, d], bits[b, d]] for d in range(3)]
            k1 = [K1[bits[a, d], bits[b, d]] for d in range(3)]
            Me[a, b] = V * m1[0] * m1[1] * m1[2]
            Ke[a, b] = alpha * V * sum(
                k1[d] * np.prod([m1[q] for q in range(3) if q != d]) / h[d] ** 2 for d in range(3))
    return Ke, Me


def interior_nodes(m):
    n = np.arange(m.n_nodes)
    i = n % (m.nx + 1)
    j = (n // (m.nx + 1)) % (m.ny + 1)
    k = n // ((m.nx + 1) * (m.ny + 1))
    return (i > 0) & (i < m.nx) & (j > 0) & (j < m.ny) & (k > 0) & (k < m.nz)


def perturbed(m, amp, seed):
    rng = np.random.default_rng(seed)
    h = min(m.lx / m.nx, m.ly / m.ny, m.lz / m.nz)
    return oracle.with_coords(m, m.X + amp * h * rng.uniform(-1, 1, m.X.shape))


def test_unit_cube_element_matrices():
    """Unit cube, alpha = 1: 12 K_ab = 4, 0, -1, -1 and 216 M_ab = 8, 4, 2, 1
    for nodes that differ in 0, 1, 2, 3 coordinates."""
    m = oracle.mesh(1, 1, 1)
    Ke, Me = op.element_matrices(m, 1.0)
    bits = corner_bits(m)
    dist = np.abs(bits[:, None, :] - bits[None, :, :]).sum(axis=2)
    assert np.abs(12 * Ke[0] - np.array([4.0, 0.0, -1.0, -1.0])[dist]).max() <= 1e-13
    assert np.abs(216 * Me[0] - np.array([8.0, 4.0, 2.0, 1.0])[dist]).max() <= 1e-13


@pytest.mark.parametrize("alpha", [1.0, 2.7])
def test_box_cell_tensor_product(alpha):
    """Anisotropic cells of a 3x2x4 mesh on a 1.5 x 1.6 x 0.4 box: every
    cell's matrices equal the tensor-product closed form (2x2x2 Gauss is
    exact for these polynomial integrands)."""
    m = oracle.mesh(3, 2, 4, 1.5, 1.6, 0.4)
    Ke, Me = op.element_matrices(m, alpha)
    h = np.array([1.5 / 3, 1.6 / 2, 0.4 / 4])
    for e in (0, 5, m.n_cells - 1):
        Kr, Mr = tensor_product_matrices(corner_bits(m, e), h, alpha)
        assert np.abs(Ke[e] - Kr).max() <= 1e-13 * np.abs(Kr).max()
        assert np.abs(Me[e] - Mr).max() <= 1e-13 * np.abs(Mr).max()


def test_matrix_free_equals_assembled():
    """Matrix-free apply / load vs the assembled matrices, with and without
    the boundary condition (constrained entries removed, y_c = x_c, F_c = 0)."""
    m = perturbed(oracle.mesh(4, 3, 3, 1.0, 1.0, 0.5), 0.2, 3)
    rng = np.random.default_rng(5)
    x, th = rng.standard_normal(m.n_nodes), rng.standard_normal(m.n_nodes)
    A, M = op.assemble(m, 1.7)
    assert np.abs(op.apply(m, 1.7, x) - A @ x).max() <= 1e-12 * np.abs(A @ x).max()
    assert np.abs(op.load(m, th) - M @ th).max() <= 1e-14 * np.abs(M @ th).max()
    mask = inputs.boundary_nodes(m.nx, m.ny, m.nz)
    c = mask == 1
    xf = np.where(c, 0.0, x)
    y = op.apply(m, 1.7, x, mask)
    ref = A @ xf
    assert np.abs(y[~c] - ref[~c]).max() <= 1e-12 * np.abs(ref).max()
    assert np.array_equal(y[c], x[c])
    F = op.load(m, th, mask)
    assert np.all(F[c] == 0.0) and np.abs(F[~c] - (M @ th)[~c]).max() <= 1e-14 * np.abs(F).max()


def test_stiffness_nullspace_symmetry_and_mass_volume():
    """On a distorted mesh: A symmetric, A 1 = 0 (constants carry no
    gradient), A positive semi-definite; M symmetric positive definite with
    1^T M 1 = volume of the (perturbed) box, the sum of the cell volumes."""
    m = perturbed(oracle.mesh(3, 3, 2, 1.0, 1.0, 0.2), 0.25, 9)
    A, M = op.assemble(m, 1.0)
    Ad, Md = A.toarray(), M.toarray()
    assert np.abs(Ad - Ad.T).max() <= 1e-14 * np.abs(Ad).max()
    assert np.abs(Ad @ np.ones(m.n_nodes)).max() <= 1e-13 * np.abs(Ad).max()
    assert np.linalg.eigvalsh(Ad).min() >= -1e-12 * np.abs(Ad).max()
    assert np.linalg.eigvalsh(Md).min() > 0
    vol = sum(indep.hex_volume(m.X[m.conn[e]]) for e in range(m.n_cells))
    assert abs(Md.sum() - vol) <= 1e-13 * vol


def test_patch_test_linear_field():
    """u = c + g . x has a constant gradient, so every interior row of A u
    vanishes on a distorted mesh."""
    m = perturbed(oracle.mesh(4, 4, 3, 1.0, 1.0, 0.3), 0.2, 21)
    g = np.array([0.3, -1.1, 2.0])
    u = 0.7 + m.X @ g
    y = op.apply(m, 1.3, u)
    inner = interior_nodes(m)
    assert np.abs(y[~inner]).max() > 0
    assert np.abs(y[inner]).max() <= 1e-13 * np.abs(y[~inner]).max()


def test_manufactured_solution_second_order():
    """u* = sin(pi x/lx) sin(pi y/ly) sin(pi z/lz) solves Eq. (24) with
    b = alpha pi^2 (lx^-2 + ly^-2 + lz^-2) u* and u* = 0 on the boundary; the
    nodal error of the discrete solution falls by ~4x per mesh halving."""
    L = np.array([1.0, 1.0, 0.2])
    alpha = 1.5
    errs = []
    for n in (4, 8, 16):
        m = oracle.mesh(n, n, n, *L)
        prob = op.Problem(m, alpha, inputs.boundary_nodes(n, n, n))
        us = np.prod(np.sin(np.pi * m.X / L), axis=1)
        theta = alpha * np.pi ** 2 * np.sum(1.0 / L ** 2) * us
        errs.append(np.abs(prob.solve(theta) - us).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 0.01
    assert np.all(rates > 1.8), rates


def test_rel_l2_error_closed_form():
    """The L2 norm of finite-element fields: with u_true = 1 + x and
    u_pred - u_true = x (both exactly representable) on a box of length lx,
    the error is sqrt((lx^3/3) / (lx + lx^2 + lx^3/3))."""
    lx = 1.3
    m = oracle.mesh(5, 3, 2, lx, 0.7, 0.2)
    prob = op.Problem(m, 1.0, inputs.boundary_nodes(5, 3, 2))
    x = m.X[:, 0]
    ref = np.sqrt((lx ** 3 / 3) / (lx + lx ** 2 + lx ** 3 / 3))
    assert abs(prob.rel_l2_error(1 + 2 * x, 1 + x) - ref) <= 1e-13


def _small_case(seed=3):
    m = perturbed(oracle.mesh(4, 4, 3, 1.0, 1.0, 0.2), 0.15, seed)
    mask = inputs.boundary_nodes(4, 4, 3)
    prob = op.Problem(m, 1.2, mask)
    rng = np.random.default_rng(seed)
    obs = np.sort(rng.choice(np.flatnonzero(mask == 0), 6, replace=False))
    U_obs = rng.standard_normal(obs.size) * 0.01
    theta = rng.standard_normal(m.n_nodes)
    return m, prob, obs, U_obs, theta


def test_gradient_equals_exact_central_differences():
    """J is quadratic in theta, so a central difference with any step is the
    exact directional derivative: compare every component of the adjoint
    gradient with (J(theta + e_i) - J(theta - e_i)) / 2."""
    m, prob, obs, U_obs, theta = _small_case()
    J, g, _, _ = prob.gradient(theta, obs, U_obs)
    fd = np.zeros(m.n_nodes)
    for i in range(m.n_nodes):
        e = np.zeros(m.n_nodes)
        e[i] = 1.0
        fd[i] = (prob.objective(theta + e, obs, U_obs)[0] - prob.objective(theta - e, obs, U_obs)[0]) / 2
    assert np.abs(g - fd).max() <= 1e-9 * np.abs(fd).max()
    # boundary values of theta only enter through the free rows of M theta
    assert np.abs(g).max() > 0


def test_taylor_remainders_rates_and_closed_form():
    """Eqs. (27)-(28) at h = 1e-4 .. 1e-1: r_zeroth ~ h, r_first ~ h^2.  Since
    U is linear in theta, r_first(h) = h^2 |U(dtheta)[obs]|^2 exactly."""
    m, prob, obs, U_obs, theta = _small_case(seed=8)
    dtheta = np.random.default_rng(81).standard_normal(m.n_nodes)
    hs = np.array([1e-4, 1e-3, 1e-2, 1e-1])
    r0, r1 = op.taylor_remainders(prob, theta, dtheta, obs, U_obs, hs)
    s0 = np.diff(np.log10(r0)) / np.diff(np.log10(hs))
    s1 = np.diff(np.log10(r1)) / np.diff(np.log10(hs))
    assert np.all(np.abs(s0 - 1) < 0.1), s0
    assert np.all(np.abs(s1 - 2) < 0.05), s1
    q = prob.solve(dtheta)[obs]
    assert np.allclose(r1 / hs ** 2, q @ q, rtol=1e-5)


def _read_paper_errors():
    out = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "poisson_inference_errors.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[int(k)] = float(v)
    return out


def test_inference_matches_paper_trend():
    """Full-field inference at the paper's size (50x50x10 on 1 x 1 x 0.2):
    the objective drops by > 1e4 within 20 L-BFGS iterations, and the
    relative L2 errors with 250 and 2500 observed points are within a factor
    of two of the printed 12.0% and 1.4% (the source centres are a reading)."""
    paper = _read_paper_errors()
    errs = {}
    for n_obs in (250, 2500):
        w = inputs.poisson_inference(n_obs=n_obs)
        m, prob = op.from_workload(w)
        U = prob.solve(w.theta_true)
        hist = []
        th = op.infer(prob, w.obs, U[w.obs], np.zeros(m.n_nodes), maxiter=20, history=hist)
        assert min(hist) < 1e-4 * hist[0]
        errs[n_obs] = prob.rel_l2_error(prob.solve(th), U)
    for n_obs, e in errs.items():
        assert paper[n_obs] / 2 <= e <= paper[n_obs] * 2, (n_obs, e)
    assert errs[2500] < errs[250] / 4
