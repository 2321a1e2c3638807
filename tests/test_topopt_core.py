"""CPU checks of the CUDA library's topology-optimisation arithmetic
(csrc/topopt_core.cuh, compiled here with g++ through
tests/topopt_core_host.cpp): the cone filter against the oracle's filter
matrix, and MMA steps (the library's per-variable formulas and dual search)
against the oracle's MMA, step by step, and in the closed-form problems."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import topopt as ot
from paper_2212_00964_gb300 import inputs
from tests import host_build


@pytest.fixture(scope="module")
def core():
    L = host_build.build("topopt_core_host", extra_flags=['-ffp-contract=off'])
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    L.host_filter.argtypes = [P, P, I, I, I, D]
    L.host_mma_step.argtypes = [I64, P, D, P, P, D, D, I, P, P, P, P, P]
    L.host_mma_step.restype = D
    L.host_filter_t.argtypes = [P, P, I, I, I, D]
    L.host_oc_step.argtypes = [I64, P, P, P, D, D, D, D, P]
    L.host_oc_step.restype = D
    return L


def p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@pytest.mark.parametrize("rmin", [1.0, 1.5, 2.3, 3.0])
def test_filter_matches_oracle(core, rmin):
    nx, ny, nz = 7, 4, 3
    g = np.random.default_rng(int(rmin * 10)).standard_normal(nx * ny * nz)
    out = np.zeros_like(g)
    core.host_filter(p(g), p(out), nx, ny, nz, rmin)
    ref = ot.filter_sensitivities(ot.filter_matrix(nx, ny, nz, rmin), g)
    assert np.abs(out - ref).max() <= 1e-14 * np.abs(ref).max()


class HostMMA:
    def __init__(self, core, n, x_min, x_max):
        self.core, self.x_min, self.x_max = core, x_min, x_max
        self.x1, self.x2, self.L, self.U = (np.zeros(n) for _ in range(4))
        self.k = 0

    def step(self, x, f0, df0, f1, df1):
        y = np.zeros_like(x)
        x = np.ascontiguousarray(x, np.float64)
        df0 = np.ascontiguousarray(df0, np.float64)
        df1 = np.ascontiguousarray(df1, np.float64)
        lam = self.core.host_mma_step(x.size, p(x), f1, p(df0), p(df1), self.x_min, self.x_max, self.k,
                                      p(self.x1), p(self.x2), p(self.L), p(self.U), p(y))
        assert lam >= 0
        self.k += 1
        self.lam = lam
        return y


def test_mma_steps_match_oracle_on_the_cantilever_loop(core):
    """Ten design iterations of the box cantilever: the oracle's loop with
    its MMA replaced by the library's arithmetic stays with the oracle's own
    loop to rounding."""
    w = inputs.topopt_cantilever(nx=8, ny=4, nz=4, lx=2.0, ly=1.0, lz=1.0)
    m = oracle.mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    mat = oracle.Material(oracle.SIMP, w.E, w.nu, w.simp_p, w.simp_emin)
    H = ot.filter_matrix(w.nx, w.ny, w.nz, 1.5)
    ref_mma = ot.MMA(m.n_cells, 0.0, 1.0)
    host_mma = HostMMA(core, m.n_cells, 0.0, 1.0)
    theta = np.full(m.n_cells, 0.5)
    for it in range(10):
        c, g, _ = ot.compliance_and_gradient(m, mat, w.mask, w.point_load, theta)
        gf = ot.filter_sensitivities(H, g)
        args = (theta, c, gf, float(theta.mean() - 0.5), np.full(m.n_cells, 1.0 / m.n_cells))
        t_ref = ref_mma.step(*args)
        t_host = host_mma.step(*args)
        assert np.abs(t_host - t_ref).max() <= 1e-12, it
        assert abs(host_mma.lam - ref_mma.lam) <= 1e-12 * max(1.0, ref_mma.lam)
        theta = t_ref


def test_mma_closed_form_nonlinear_constraint(core):
    b = np.array([61.0, 37.0, 19.0, 7.0, 1.0])
    a = 0.0624
    lam = ((a / 3) ** 0.75 * np.sum(b ** 0.25)) ** (4 / 3)
    xs = (3 * lam * b / a) ** 0.25
    mma = HostMMA(core, 5, 1.0, 10.0)
    x = np.full(5, 5.0)
    for _ in range(60):
        x = mma.step(x, a * x.sum(), np.full(5, a), np.sum(b / x ** 3) - 1, -3 * b / x ** 4)
    assert np.abs(x - xs).max() <= 1e-9 * xs.max()


@pytest.mark.parametrize("rmin", [1.0, 1.5, 2.3])
def test_filter_transpose_matches_oracle(core, rmin):
    nx, ny, nz = 6, 5, 3
    g = np.random.default_rng(int(rmin * 7)).standard_normal(nx * ny * nz)
    out = np.zeros_like(g)
    core.host_filter_t(p(g), p(out), nx, ny, nz, rmin)
    ref = ot.filter_transpose(ot.filter_matrix(nx, ny, nz, rmin), g)
    assert np.abs(out - ref).max() <= 1e-14 * np.abs(ref).max()


def test_oc_steps_match_oracle(core):
    rng = np.random.default_rng(23)
    n = 40
    c = rng.uniform(0.2, 1.0, n)
    dv = rng.uniform(0.5, 1.5, n)
    x = np.full(n, 0.4)
    for _ in range(8):
        g = -c / x ** 2
        ref, lam_ref = ot.oc_step(x, g, dv, 0.4, 0.15, 0.01, 1.0)
        y = np.zeros(n)
        lam = core.host_oc_step(n, p(x), p(np.ascontiguousarray(g)), p(dv), 0.4, 0.15, 0.01, 1.0, p(y))
        assert abs(lam - lam_ref) <= 1e-12 * lam_ref
        assert np.abs(y - ref).max() <= 1e-12
        x = ref


def test_edge_cases(core):
    """Filters on one-cell-thick boxes and a single cell; OC with zero and
    positive gradient entries (those variables go to their lower limit);
    MMA on a variable already at its bound with a gradient pushing outward
    (it stays there)."""
    for nx, ny, nz in ((1, 1, 1), (7, 1, 1), (1, 5, 1), (4, 3, 1)):
        g = np.random.default_rng(nx * 10 + ny).standard_normal(nx * ny * nz)
        H = ot.filter_matrix(nx, ny, nz, 2.0)
        out = np.zeros_like(g)
        core.host_filter(p(g), p(out), nx, ny, nz, 2.0)
        assert np.abs(out - ot.filter_sensitivities(H, g)).max() <= 1e-14 * max(1.0, np.abs(g).max())
        core.host_filter_t(p(g), p(out), nx, ny, nz, 2.0)
        assert np.abs(out - ot.filter_transpose(H, g)).max() <= 1e-14 * max(1.0, np.abs(g).max())
    x = np.array([0.5, 0.5, 0.5, 0.5])
    g = np.array([-1.0, 0.0, 2.0, -3.0])
    y = np.zeros(4)
    core.host_oc_step(4, p(x), p(g), p(np.ones(4)), 0.3, 0.2, 0.0, 1.0, p(y))
    ref, _ = ot.oc_step(x, g, np.ones(4), 0.3, 0.2, 0.0, 1.0)
    assert np.abs(y - ref).max() <= 1e-12 and y[1] == 0.3 and y[2] == 0.3
    mma = HostMMA(core, 2, 0.0, 1.0)
    x = np.array([1.0, 0.0])
    for _ in range(3):
        x = mma.step(x, 0.0, np.array([-1.0, 1.0]), -1.0, np.zeros(2))
    assert np.array_equal(x, [1.0, 0.0])


def test_mma_infeasible_constraint_reports_no_multiplier(core):
    """x >= 2 with x <= 1 (f1 = 2 - x): no multiplier makes the subproblem
    feasible, so the dual search returns a negative value (the library
    reports FEM_ERR_NOT_CONVERGED) and leaves the state untouched."""
    x = np.array([0.5, 0.7])
    x1, x2, lo, up, y = (np.zeros(2) for _ in range(5))
    lam = core.host_mma_step(2, p(x), float(2 - x.mean()), p(np.zeros(2)), p(np.full(2, -0.5)), 0.0, 1.0, 0,
                             p(x1), p(x2), p(lo), p(up), p(y))
    assert lam < 0 and np.all(x1 == 0) and np.all(y == 0)


def test_mma_first_step_stops_at_the_move_limits(core):
    """In the first step the asymptotes sit 0.5 of the range away and the
    move limits 9/10 of the way to them: a linear objective with a slack
    constraint moves every variable by 0.45 of the range, as in the oracle."""
    mma = HostMMA(core, 3, 0.0, 2.0)
    y = mma.step(np.full(3, 1.0), 0.0, np.array([1.0, -1.0, 2.0]), -5.0, np.zeros(3))
    assert np.abs(y - [0.1, 1.9, 0.1]).max() <= 1e-15
