"""Pins of the topology-optimisation oracle (Sec. 3.2): the sensitivity
filter against a library convolution, the MMA step against closed-form
optima (with and without active bounds, linear and nonlinear constraints),
and the design loop on the box cantilever against what the mathematics
fixes (active volume constraint, full solid as the lower bound)."""
import numpy as np
import pytest
from scipy import ndimage, optimize

import oracle
from oracle import topopt as ot
from paper_2212_00964_gb300 import inputs


@pytest.mark.parametrize("rmin", [1.5, 2.3])
def test_filter_equals_normalised_library_convolution(rmin):
    """The filter on a structured grid is a correlation with the cone kernel
    max(0, r - |d|) (zero outside the box), divided by the same correlation
    of ones: scipy.ndimage.correlate gives both."""
    nx, ny, nz = 5, 4, 3
    H = ot.filter_matrix(nx, ny, nz, rmin)
    g = np.random.default_rng(1).standard_normal(nx * ny * nz)
    R = int(np.ceil(rmin))
    d = np.arange(-R, R + 1)
    DK, DJ, DI = np.meshgrid(d, d, d, indexing="ij")
    kern = np.maximum(0.0, rmin - np.sqrt(DI ** 2 + DJ ** 2 + DK ** 2))
    G = g.reshape(nz, ny, nx)  # cell id = i + nx (j + ny k)
    num = ndimage.correlate(G, kern, mode="constant", cval=0.0)
    den = ndimage.correlate(np.ones_like(G), kern, mode="constant", cval=0.0)
    ref = (num / den).reshape(-1)
    assert np.abs(ot.filter_sensitivities(H, g) - ref).max() <= 1e-14 * np.abs(ref).max()


def test_filter_identity_and_constants():
    H = ot.filter_matrix(4, 3, 2, 1.0)
    g = np.random.default_rng(2).standard_normal(24)
    assert np.array_equal(ot.filter_sensitivities(H, g), g)
    H = ot.filter_matrix(4, 3, 2, 2.0)
    assert np.abs(ot.filter_sensitivities(H, np.full(24, 3.7)) - 3.7).max() <= 1e-15 * 3.7
    assert abs(H - H.T).max() == 0


def run_mma(x0, fun, n_iter, x_min, x_max):
    mma = ot.MMA(x0.size, x_min, x_max)
    x = x0.copy()
    for _ in range(n_iter):
        f0, df0, f1, df1 = fun(x)
        x = mma.step(x, f0, df0, f1, df1)
        assert mma.lam >= 0 and np.all(x >= x_min) and np.all(x <= x_max)
    return x


def test_mma_reciprocal_objective_with_active_bounds():
    """min sum c_j / x_j s.t. mean(x) <= V, x in [0.01, 1]: by the KKT
    conditions x_j = min(1, sqrt(c_j / (n lam))) with lam fixed by the
    active constraint (found here with brentq)."""
    rng = np.random.default_rng(3)
    n, V = 16, 0.45
    c = rng.uniform(0.2, 1.0, n)
    c[:3] = 30.0  # these want x > 1 and sit on the bound
    xs_of = lambda lam: np.clip(np.sqrt(c / (n * lam)), 0.01, 1.0)
    lam = optimize.brentq(lambda t: xs_of(t).mean() - V, 1e-8, 1e8, xtol=1e-300, rtol=1e-15)
    xs = xs_of(lam)
    assert np.all(xs[:3] == 1.0) and np.all(xs[3:] < 1.0)

    def fun(x):
        return np.sum(c / x), -c / x ** 2, x.mean() - V, np.full(n, 1.0 / n)

    x = run_mma(np.full(n, V), fun, 80, 0.01, 1.0)
    assert np.abs(x - xs).max() <= 1e-9


def test_mma_nonlinear_constraint_closed_form():
    """min a sum x s.t. sum b_j / x_j^3 <= 1: x_j = (3 lam b_j / a)^(1/4) with
    lam^(3/4) = (a/3)^(3/4) sum b_j^(1/4) (Lagrange conditions)."""
    b = np.array([61.0, 37.0, 19.0, 7.0, 1.0])
    a = 0.0624
    lam = ((a / 3) ** 0.75 * np.sum(b ** 0.25)) ** (4 / 3)
    xs = (3 * lam * b / a) ** 0.25

    def fun(x):
        return a * x.sum(), np.full(5, a), np.sum(b / x ** 3) - 1, -3 * b / x ** 4

    x = run_mma(np.full(5, 5.0), fun, 60, 1.0, 10.0)
    assert np.abs(x - xs).max() <= 1e-9 * xs.max()


def test_mma_inactive_constraint_reaches_bounds():
    """With a slack constraint the objective alone decides: a linear
    objective drives every variable to its bound within a few steps."""
    def fun(x):
        return float(np.sum(x * [1, -1, 2])), np.array([1.0, -1.0, 2.0]), -5.0, np.zeros(3)

    x = run_mma(np.full(3, 0.5), fun, 40, 0.0, 1.0)
    assert np.abs(x - [0.0, 1.0, 0.0]).max() <= 1e-6


def test_mma_first_step_stops_at_move_limits():
    """In the first iteration the asymptotes sit s0 = 0.5 of the range away
    and the move limits 9/10 of the way to them, so a linear objective with a
    slack constraint moves each variable by exactly 0.45 of the range."""
    def fun(x):
        return 0.0, np.array([1.0, -1.0, 2.0]), -5.0, np.zeros(3)

    mma = ot.MMA(3, 0.0, 2.0)
    x = mma.step(np.full(3, 1.0), *fun(None))
    assert np.abs(x - [0.1, 1.9, 0.1]).max() <= 1e-15


def test_design_loop_filter_smooths_the_design():
    """A filter radius wider than the box averages the sensitivities, so the
    design stays smooth: after 10 iterations its total variation is far
    below that of the unfiltered loop (radius 1 = identity filter)."""
    w = inputs.topopt_cantilever()
    m = oracle.mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    mat = oracle.Material(oracle.SIMP, w.E, w.nu, w.simp_p, w.simp_emin)

    def tv(th):
        T = th.reshape(w.nz, w.ny, w.nx)
        return sum(np.abs(np.diff(T, axis=a)).sum() for a in range(3))

    t_raw = tv(ot.optimise(m, mat, w.mask, w.point_load, 0.5, 1.0, 10))
    t_wide = tv(ot.optimise(m, mat, w.mask, w.point_load, 0.5, 100.0, 10))
    assert t_wide < 0.1 * t_raw


def test_design_loop_on_box_cantilever():
    """40 iterations on the 16x8x4 cantilever: the volume constraint is
    active (mean theta = 0.5), the compliance falls far below the uniform
    design's and stays above the full solid's (half the material cannot be
    stiffer than all of it), the uniform start has c = c_full / 0.5^p up to
    the stiffness floor, and the design is nearly black and white."""
    w = inputs.topopt_cantilever()
    m = oracle.mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    mat = oracle.Material(oracle.SIMP, w.E, w.nu, w.simp_p, w.simp_emin)
    hist = []
    th = ot.optimise(m, mat, w.mask, w.point_load, w.extra["volfrac"], w.extra["rmin"], 40, history=hist)
    c_full = ot.compliance_and_gradient(m, mat, w.mask, w.point_load, np.ones(m.n_cells))[0]
    c_end = ot.compliance_and_gradient(m, mat, w.mask, w.point_load, th)[0]
    c0 = hist[0][0]
    e_half = w.simp_emin + 0.5 ** w.simp_p * (1 - w.simp_emin)
    assert abs(c0 - c_full / e_half) <= 1e-9 * c0
    assert abs(th.mean() - 0.5) <= 1e-4
    assert c_full < c_end < c0 / 4
    assert np.mean((th > 0.1) & (th < 0.9)) < 0.1
    cs = np.array([h[0] for h in hist])
    assert np.all(np.diff(cs[:12]) < 0)


def test_filter_transpose_is_the_adjoint():
    """<F a, b> = <a, F^T b> for the normalised filter F = diag(1/Hs) H, and
    the chain rule through a density filter matches central differences."""
    nx, ny, nz = 5, 4, 3
    H = ot.filter_matrix(nx, ny, nz, 1.7)
    rng = np.random.default_rng(21)
    a, b = rng.standard_normal(60), rng.standard_normal(60)
    assert abs(ot.filter_sensitivities(H, a) @ b - a @ ot.filter_transpose(H, b)) <= 1e-13 * np.abs(a).sum()
    # J(theta) = sum c_e / filter(theta)_e
    c = rng.uniform(0.5, 1.5, 60)
    theta = rng.uniform(0.3, 0.9, 60)
    J = lambda t: np.sum(c / ot.filter_sensitivities(H, t))
    g_tilde = -c / ot.filter_sensitivities(H, theta) ** 2
    g = ot.filter_transpose(H, g_tilde)
    h = 1e-6
    for e in (0, 17, 59):
        d = np.zeros(60)
        d[e] = h
        assert abs((J(theta + d) - J(theta - d)) / (2 * h) - g[e]) <= 1e-6 * np.abs(g).max()


def test_oc_reaches_the_closed_form_optimum():
    """min sum c_j / x_j s.t. mean(x) <= V: the OC fixed point is the KKT
    point x_j = V n sqrt(c_j) / sum sqrt(c) (all inside the bounds here), and
    the volume constraint holds with equality at every step."""
    rng = np.random.default_rng(22)
    n, V = 30, 0.4
    c = rng.uniform(0.2, 1.0, n)
    xs = V * n * np.sqrt(c) / np.sqrt(c).sum()
    x = np.full(n, V)
    dv = np.ones(n)
    for _ in range(60):
        x, lam = ot.oc_step(x, -c / x ** 2, dv, V, move=0.2, x_min=0.01)
        assert abs(x.mean() - V) <= 1e-10
    assert np.abs(x - xs).max() <= 1e-9


def test_oc_move_limit_and_bounds():
    x = np.array([0.5, 0.5, 0.05, 0.95])
    g = np.array([-100.0, -1e-6, -1.0, -1.0])
    y, _ = ot.oc_step(x, g, np.ones(4), 0.5, move=0.1, x_min=0.0, x_max=1.0)
    assert np.all(y >= np.maximum(0, x - 0.1) - 1e-15) and np.all(y <= np.minimum(1, x + 0.1) + 1e-15)
    assert y[0] == 0.6 and y[1] == 0.4


def test_hyperelastic_simp_gradient_central_differences():
    """SIMP on the Neo-Hookean law (the paper's plate): the chain-ruled
    adjoint gradient against central differences of the compliance, and the
    small-load limit where it matches the linear-elastic SIMP gradient."""
    w = inputs.topopt_cantilever(nx=4, ny=4, nz=4, lx=2.0, ly=1.0, lz=1.0)
    m = oracle.mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    rng = np.random.default_rng(41)
    theta = rng.uniform(0.3, 1.0, m.n_cells)
    f = w.point_load * 2e-3  # tip deflection of a few percent of the depth: mildly nonlinear
    c, g, _ = ot.compliance_and_gradient_nh(m, 1.0, 0.3, w.mask, f, theta)
    h = 1e-6
    for e in (0, 21, 42, 63):
        tp, tm = theta.copy(), theta.copy()
        tp[e] += h
        tm[e] -= h
        fd = (ot.compliance_and_gradient_nh(m, 1.0, 0.3, w.mask, f, tp)[0] -
              ot.compliance_and_gradient_nh(m, 1.0, 0.3, w.mask, f, tm)[0]) / (2 * h)
        assert abs(fd - g[e]) <= 1e-5 * np.abs(g).max()
    # tiny load: the hyperelastic compliance gradient approaches the linear one
    mat = oracle.Material(oracle.SIMP, 1.0, 0.3, 3.0, 1e-3)
    f_small = w.point_load * 1e-6
    _, g_nh, _ = ot.compliance_and_gradient_nh(m, 1.0, 0.3, w.mask, f_small, theta, rtol=1e-8)
    _, g_le, _ = ot.compliance_and_gradient(m, mat, w.mask, f_small, theta)
    assert np.abs(g_nh - g_le).max() <= 1e-4 * np.abs(g_le).max()
