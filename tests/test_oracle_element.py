"""Pins of the oracle's element level: shape functions, Gauss rule, geometry,
linear-elastic element stiffness, constitutive laws (Sec. 2.3, Eqs. (11), (13))."""
import numpy as np
import pytest

import oracle
from tests import indep

RNG = np.random.default_rng(1234)


def test_shape_partition_of_unity_and_nodality():
    for _ in range(20):
        xi = RNG.uniform(-1, 1, 3)
        N, dN = oracle.shape(*xi)
        assert abs(N.sum() - 1) < 1e-15
        assert np.abs(dN.sum(axis=0)).max() < 1e-15
    for b in range(8):
        N, _ = oracle.shape(*indep.CORNERS[b])
        assert np.allclose(N, np.eye(8)[b], atol=0)
    # derivative by central differences
    xi = RNG.uniform(-0.5, 0.5, 3)
    _, dN = oracle.shape(*xi)
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1e-6
        Np, _ = oracle.shape(*(xi + e))
        Nm, _ = oracle.shape(*(xi - e))
        assert np.allclose((Np - Nm) / 2e-6, dN[:, k], atol=1e-9)


def test_gauss_rule_exact_for_cubic_per_direction():
    gp, w = oracle.gauss()
    assert abs(w.sum() - 8) < 1e-14
    # int_{[-1,1]^3} x^a y^b z^c = prod (2/(p+1) if p even else 0), p <= 3 exact
    for a in range(4):
        for b in range(4):
            for c in range(4):
                exact = np.prod([2 / (p + 1) if p % 2 == 0 else 0.0 for p in (a, b, c)])
                got = np.sum(w * gp[:, 0] ** a * gp[:, 1] ** b * gp[:, 2] ** c)
                assert abs(got - exact) < 1e-14
    # xi fastest
    assert gp[0, 0] < 0 < gp[1, 0] and gp[0, 1] == gp[1, 1]


def test_volume_of_affine_cells():
    m = oracle.mesh(2, 2, 2, 1.0, 2.0, 3.0)
    A = np.array([[1.0, 0.2, 0.1], [0.0, 1.1, -0.3], [0.05, 0.0, 0.9]])
    Xa = m.X @ A.T
    ma = oracle.with_coords(m, Xa)
    # body force b = 1 in x integrates to sum_a f_a = volume
    f = oracle.body_force(ma, np.tile([1.0, 0, 0], (m.n_cells, 8, 1)))
    assert abs(f[0::3].sum() - 6.0 * np.linalg.det(A)) < 1e-12


@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (0.5, 0.25, 2.0)])
def test_le_element_stiffness_matches_voigt(h):
    hx, hy, hz = h
    m = oracle.mesh(1, 1, 1, hx, hy, hz)
    mat = oracle.Material(oracle.LINEAR, 70e3, 0.3)
    Ke = oracle.element_tangent(m, mat, np.zeros(m.n_dofs), 0)
    Kv = indep.voigt_ke(hx, hy, hz, 70e3, 0.3)
    assert np.abs(Ke - Kv).max() <= 1e-10 * np.abs(Kv).max()
    assert np.abs(Ke - Ke.T).max() <= 1e-12 * np.abs(Ke).max()
    ev = np.linalg.eigvalsh(Ke)
    assert np.sum(np.abs(ev) < 1e-9 * ev.max()) == 6
    assert np.all(ev > -1e-9 * ev.max())
    R = indep.rigid_modes(m.X[m.conn[0]])
    assert np.abs(Ke @ R.T).max() < 1e-9 * np.abs(Ke).max()


def test_le_stress_is_voigt_law():
    H = RNG.standard_normal((3, 3)) * 0.01
    P, _ = oracle.stress(oracle.LINEAR, 70e3, 0.3, H)
    eps = 0.5 * (H + H.T)
    v = np.array([eps[0, 0], eps[1, 1], eps[2, 2], 2 * eps[1, 2], 2 * eps[0, 2], 2 * eps[0, 1]])
    s = indep.voigt_D(70e3, 0.3) @ v
    S = np.array([[s[0], s[5], s[4]], [s[5], s[1], s[3]], [s[4], s[3], s[2]]])
    assert np.allclose(P, S, rtol=1e-13, atol=1e-12)


def test_nh_stress_zero_at_identity():
    P, J = oracle.stress(oracle.NEOHOOKE, 10.0, 0.3, np.zeros((3, 3)))
    assert np.abs(P).max() < 1e-15 and J == 1.0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_nh_stress_is_energy_gradient(seed):
    rng = np.random.default_rng(seed)
    H = 0.2 * rng.standard_normal((3, 3))
    E, nu = 10.0, 0.3
    P, J = oracle.stress(oracle.NEOHOOKE, E, nu, H)
    assert J > 0
    Pfd = indep.fd_grad(lambda Fm: indep.nh_energy(Fm, E, nu), np.eye(3) + H, h=1e-5)
    assert np.abs(P - Pfd).max() <= 1e-8 * np.abs(P).max()


def test_nh_frame_indifference():
    rng = np.random.default_rng(5)
    H = 0.2 * rng.standard_normal((3, 3))
    Q = indep.random_rotation(rng)
    P, _ = oracle.stress(oracle.NEOHOOKE, 10.0, 0.3, H)
    F = np.eye(3) + H
    PQ, _ = oracle.stress(oracle.NEOHOOKE, 10.0, 0.3, Q @ F - np.eye(3))
    assert np.abs(PQ - Q @ P).max() <= 1e-12 * np.abs(P).max()


@pytest.mark.parametrize("kind", [oracle.LINEAR, oracle.NEOHOOKE])
def test_dstress_is_stress_derivative_and_major_symmetric(kind):
    rng = np.random.default_rng(11)
    H = 0.15 * rng.standard_normal((3, 3))
    dH = rng.standard_normal((3, 3))
    dG = rng.standard_normal((3, 3))
    E, nu = 10.0, 0.3
    dP = oracle.dstress(kind, E, nu, H, dH)
    h = 1e-6
    Pp, _ = oracle.stress(kind, E, nu, H + h * dH)
    Pm, _ = oracle.stress(kind, E, nu, H - h * dH)
    assert np.abs(dP - (Pp - Pm) / (2 * h)).max() <= 1e-7 * np.abs(dP).max()
    dQ = oracle.dstress(kind, E, nu, H, dG)
    assert abs(np.sum(dG * dP) - np.sum(dH * dQ)) <= 1e-12 * np.abs(dP).max() * 10


def test_nh_tangent_at_identity_is_linear_elasticity():
    """At F = I the Neo-Hookean tangent is the isotropic linear-elastic one
    with lambda = kappa - 2G/3 = E nu / ((1+nu)(1-2nu)) and mu = G."""
    rng = np.random.default_rng(3)
    E, nu = 10.0, 0.3
    for _ in range(5):
        dH = rng.standard_normal((3, 3))
        a = oracle.dstress(oracle.NEOHOOKE, E, nu, np.zeros((3, 3)), dH)
        b = oracle.dstress(oracle.LINEAR, E, nu, np.zeros((3, 3)), dH)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
