"""Pins of the J2 plasticity oracle (Sec. 2.3, Eqs. (14)-(15)): the return
map against the Voigt elastic law and the geometry of the radial return, its
tangent against central differences, the global tangent against the
residual, and a load/unload/reverse-yield path against the closed form of
uniaxial perfect plasticity."""
import numpy as np
import pytest

import oracle
from oracle import plasticity as pl
from paper_2212_00964_gb300 import inputs
from tests import indep

MAT = pl.Material(70e3, 0.3, 250.0)


def voigt(e):
    """Engineering Voigt vector of a symmetric strain (shear doubled)."""
    return np.array([e[0, 0], e[1, 1], e[2, 2], 2 * e[1, 2], 2 * e[0, 2], 2 * e[0, 1]])


def unvoigt_stress(s):
    return np.array([[s[0], s[5], s[4]], [s[5], s[1], s[3]], [s[4], s[3], s[2]]])


def elastic_trial(eps_old, sig_old, H):
    """sigma^{k-1} + D : (sym H - eps^{k-1}) by the Voigt matrix."""
    de = 0.5 * (H + H.T) - eps_old
    return sig_old + unvoigt_stress(indep.voigt_D(MAT.E, MAT.nu) @ voigt(de))


def mises(s):
    d = s - np.trace(s) / 3 * np.eye(3)
    return np.sqrt(1.5 * np.sum(d * d))


def random_history(rng, scale):
    e = rng.standard_normal((3, 3)) * scale
    e = 0.5 * (e + e.T)
    sig = unvoigt_stress(indep.voigt_D(MAT.E, MAT.nu) @ voigt(e))
    sig *= min(1.0, 0.9 * MAT.sy / mises(sig))  # a state inside the yield surface
    return e, sig


def test_elastic_branch_is_voigt_law():
    """Below the yield surface sigma^k is the elastic trial stress."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        eo, so = random_history(rng, 1e-3)
        H = eo + rng.standard_normal((3, 3)) * 1e-5
        sig, eps, f = pl.stress(MAT, eo, so, H)
        tr = elastic_trial(eo, so, H)
        assert f < 0
        assert np.abs(sig - tr).max() <= 1e-12 * MAT.sy
        assert np.abs(eps - 0.5 * (H + H.T)).max() == 0.0


def test_plastic_branch_radial_return_geometry():
    """Above the yield surface: Mises(sigma^k) = sigma_y, the pressure of the
    trial state is kept, and sigma_trial - sigma^k is a positive multiple of
    the trial deviator (radial return)."""
    rng = np.random.default_rng(2)
    n_plastic = 0
    for _ in range(40):
        eo, so = random_history(rng, 2e-3)
        H = eo + rng.standard_normal((3, 3)) * 5e-3
        sig, _, f = pl.stress(MAT, eo, so, H)
        tr = elastic_trial(eo, so, H)
        if mises(tr) <= MAT.sy:
            continue
        n_plastic += 1
        assert f > 0 and abs(f - (mises(tr) - MAT.sy)) <= 1e-9 * MAT.sy
        assert abs(mises(sig) - MAT.sy) <= 1e-10 * MAT.sy
        assert abs(np.trace(sig) - np.trace(tr)) <= 1e-10 * MAT.sy
        d = tr - sig
        s = tr - np.trace(tr) / 3 * np.eye(3)
        c = np.sum(d * s) / np.sum(s * s)
        assert c > 0 and np.abs(d - c * s).max() <= 1e-10 * MAT.sy
    assert n_plastic >= 20


def test_hydrostatic_increment_never_yields():
    eo, so = np.zeros((3, 3)), np.zeros((3, 3))
    for v in (1e-3, 1e-1, -1e-1):
        sig, _, f = pl.stress(MAT, eo, so, v * np.eye(3))
        assert f == -MAT.sy
        K = MAT.E / (3 * (1 - 2 * MAT.nu))
        assert np.abs(sig - 3 * K * v * np.eye(3)).max() <= 1e-12 * abs(3 * K * v)


@pytest.mark.parametrize("branch", ["elastic", "plastic"])
def test_return_map_tangent_central_differences(branch):
    """d sigma = central FD of the return map, for random directions, away
    from the yield surface."""
    rng = np.random.default_rng(3 if branch == "elastic" else 4)
    checked = 0
    for _ in range(30):
        eo, so = random_history(rng, 2e-3)
        H = eo + rng.standard_normal((3, 3)) * (1e-5 if branch == "elastic" else 5e-3)
        f = pl.stress(MAT, eo, so, H)[2]
        if (f < 0) != (branch == "elastic") or abs(f) < 1e-3 * MAT.sy:
            continue
        checked += 1
        dH = rng.standard_normal((3, 3))
        h = 1e-8
        fd = (pl.stress(MAT, eo, so, H + h * dH)[0] - pl.stress(MAT, eo, so, H - h * dH)[0]) / (2 * h)
        ds = pl.dstress(MAT, eo, so, H, dH)
        assert np.abs(ds - fd).max() <= 1e-6 * np.abs(fd).max()
    assert checked >= 10


def test_plastic_tangent_flow_direction_and_volume():
    """On the yield surface, straining along the flow direction (the
    deviator) changes no stress; a volumetric strain gives 3 K tr I."""
    rng = np.random.default_rng(5)
    eo, so = random_history(rng, 2e-3)
    H = eo + rng.standard_normal((3, 3)) * 5e-3
    sig, _, f = pl.stress(MAT, eo, so, H)
    assert f > 0
    s = sig - np.trace(sig) / 3 * np.eye(3)
    assert np.abs(pl.dstress(MAT, eo, so, H, s)).max() <= 1e-10 * np.abs(s).max() * MAT.E
    K = MAT.E / (3 * (1 - 2 * MAT.nu))
    assert np.abs(pl.dstress(MAT, eo, so, H, np.eye(3)) - 3 * K * np.eye(3)).max() <= 1e-9 * K


def test_global_tangent_is_residual_derivative():
    """On a distorted 2x2x2 mesh with a partly yielded state: K(u) x = central
    FD of R, and the matrix-free apply equals the assembled tangent."""
    m = oracle.mesh(2, 2, 2)
    rng = np.random.default_rng(6)
    m = oracle.with_coords(m, m.X + 0.1 * 0.5 * rng.uniform(-1, 1, m.X.shape))
    hist = pl.zero_history(m)
    # a history from one elastic-plastic step, then a further state
    u1 = 1.2e-3 * rng.standard_normal(m.n_dofs)
    _, hist, n1 = pl.residual(m, MAT, hist, u1)
    u = u1 + 3e-4 * rng.standard_normal(m.n_dofs)
    _, _, n_yield = pl.residual(m, MAT, hist, u)
    assert 0 < n_yield < 8 * m.n_cells
    x = rng.standard_normal(m.n_dofs)
    h = 1e-9
    fd = (pl.residual(m, MAT, hist, u + h * x)[0] - pl.residual(m, MAT, hist, u - h * x)[0]) / (2 * h)
    y = pl.tangent_apply(m, MAT, hist, u, x)
    assert np.abs(y - fd).max() <= 1e-5 * np.abs(fd).max()
    K = pl.assemble(m, MAT, hist, u)
    assert np.abs(K @ x - y).max() <= 1e-11 * np.abs(y).max()


def test_gauss_point_weights_and_volume_average():
    """w_q det J of each cell sums to its volume (independent 3-point rule)
    on a distorted mesh; the volume average of x_q (the physical Gauss
    points) is the centroid of the box when only interior nodes move."""
    m = oracle.mesh(3, 2, 2, 1.0, 0.8, 0.6)
    rng = np.random.default_rng(12)
    X = m.X.copy()
    inner = ((X > 1e-12) & (X < np.array([1.0, 0.8, 0.6]) - 1e-12)).all(axis=1)
    X[inner] += 0.05 * rng.uniform(-1, 1, (inner.sum(), 3))
    m = oracle.with_coords(m, X)
    w = pl.gp_jxw(m)
    for e in range(m.n_cells):
        assert abs(w[e].sum() - indep.hex_volume(m.X[m.conn[e]])) <= 1e-14
    xg = oracle.gauss_points_phys(m)
    assert np.abs(pl.volume_average(m, xg) - np.array([0.5, 0.4, 0.3])).max() <= 1e-14


def uniaxial_closed_form(strains, E, sy):
    """Uniaxial perfect plasticity, strain-driven: sigma_k = clip(sigma_{k-1}
    + E (eps_k - eps_{k-1}), -sy, sy); plastic strain eps - sigma/E."""
    sig, prev, out = 0.0, 0.0, []
    for e in strains:
        sig = float(np.clip(sig + E * (e - prev), -sy, sy))
        prev = e
        out.append(sig)
    return np.array(out)


def test_uniaxial_load_unload_reverse_yield_closed_form():
    """The load/unload path of the plasticity example on a box with symmetry
    rollers: the state is uniaxial stress, so at every step the
    volume-averaged sigma_zz, the lateral strain -nu sigma/E - eps_p/2 and
    sigma_xx = 0 follow the 1D closed form (radial return is exact for this
    proportional path), through yield, elastic unloading and reverse yield."""
    n, L = 2, 1.0
    mask, ubars, strains, (E, nu, sy) = inputs.j2_uniaxial(n=n, L=L)
    mat = pl.Material(E, nu, sy)
    m = oracle.mesh(n, n, n, L, L, L)
    res = pl.solve_path(m, mat, mask, ubars)
    ref = uniaxial_closed_form(strains, E, sy)
    x1 = inputs.face_nodes(n, n, n, "x1")
    for k, (u, (eps, sig), n_yield) in enumerate(res):
        avg = pl.volume_average(m, sig)
        assert abs(avg[2, 2] - ref[k]) <= 1e-9 * sy, (k, avg[2, 2], ref[k])
        assert np.abs(avg - np.diag([0, 0, ref[k]])).max() <= 1e-9 * sy
        # homogeneous: every Gauss point carries the average
        assert np.abs(sig - avg).max() <= 1e-9 * sy
        ep = strains[k] - ref[k] / E
        lat = -nu * ref[k] / E - ep / 2
        assert np.abs(u[3 * x1] - L * lat).max() <= 1e-12
        trial = (ref[k - 1] if k else 0.0) + E * (strains[k] - (strains[k - 1] if k else 0.0))
        if abs(trial) < sy * (1 - 1e-9):
            assert n_yield == 0
        elif abs(trial) > sy * (1 + 1e-9):
            assert n_yield == 8 * m.n_cells
    # the path reaches yield, unloads elastically and yields in reverse
    assert ref.max() == sy and ref.min() == -sy and np.any(np.abs(ref) < sy)
