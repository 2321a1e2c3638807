"""CPU run of the library's Poisson solves and gradient: the CG control,
the mixed-precision refinement and the objective / adjoint control
(dpcg_control.h, poisson_control.h) with the stencil rows (poisson_core.cuh)
compiled for the host through tests/poisson_solve_host.cpp, against the
oracle's LU solves and adjoint gradient (Sec. 3.1)."""
import ctypes

import numpy as np
import pytest

from oracle import poisson as op
from paper_2212_00964_gb300 import inputs
from tests import host_build


@pytest.fixture(scope="module")
def L():
    lib = host_build.build("poisson_solve_host", extra_flags=[])
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    lib.host_poisson_solve.argtypes = [I, I, I, D, D, D, D, P, P, P, D, I, I, ctypes.POINTER(I), ctypes.POINTER(D)]
    lib.host_poisson_gradient.argtypes = [I, I, I, D, D, D, D, P, P, P, P, I64, D, I, I, P, P, P,
                                          ctypes.POINTER(D), ctypes.POINTER(I)]
    lib.host_poisson_error.restype = ctypes.c_char_p
    return lib


def p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def workload():
    return inputs.poisson_inference(20, 20, 5, 1.0, 1.0, 0.2, n_obs=40, seed=2)


@pytest.mark.parametrize("mixed", [0, 1])
def test_solve_matches_lu(L, mixed):
    w = workload()
    m, prob = op.from_workload(w)
    b = op.load(m, w.theta_true, w.mask)
    u = np.zeros(m.n_nodes)
    it, res = ctypes.c_int(), ctypes.c_double()
    rc = L.host_poisson_solve(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz, w.alpha, p(w.mask), p(b), p(u), 1e-11, 20000,
                              mixed, ctypes.byref(it), ctypes.byref(res))
    assert rc == 0, L.host_poisson_error()
    ref = prob.solve(w.theta_true)
    assert res.value <= 1e-11
    assert np.linalg.norm(u - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("mixed", [0, 1])
def test_gradient_matches_oracle(L, mixed):
    w = workload()
    m, prob = op.from_workload(w)
    rng = np.random.default_rng(4)
    theta = rng.standard_normal(m.n_nodes)
    u_obs = 0.01 * rng.standard_normal(w.obs.size)
    J_ref, g_ref, u_ref, lam_ref = prob.gradient(theta, w.obs, u_obs)
    u, lam, g = np.zeros(m.n_nodes), np.zeros(m.n_nodes), np.zeros(m.n_nodes)
    J, its = ctypes.c_double(), (ctypes.c_int * 2)()
    obs = np.ascontiguousarray(w.obs, np.int64)
    rc = L.host_poisson_gradient(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz, w.alpha, p(w.mask), p(theta), p(obs),
                                 p(u_obs), obs.size, 1e-12, 20000, mixed, p(u), p(lam), p(g), ctypes.byref(J), its)
    assert rc == 0, L.host_poisson_error()
    assert abs(J.value - J_ref) <= 1e-9 * J_ref
    assert np.linalg.norm(g - g_ref) <= 1e-8 * np.linalg.norm(g_ref)
    assert np.linalg.norm(lam - lam_ref) <= 1e-8 * np.linalg.norm(lam_ref)
    assert its[0] > 0 and its[1] > 0


def test_bad_observation_and_iteration_limit(L):
    w = workload()
    m, _ = op.from_workload(w)
    obs = np.ascontiguousarray(w.obs, np.int64)
    obs[1] = m.n_nodes
    z = np.zeros(m.n_nodes)
    J, its = ctypes.c_double(), (ctypes.c_int * 2)()
    rc = L.host_poisson_gradient(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz, w.alpha, p(w.mask), p(np.ones(m.n_nodes)),
                                 p(obs), p(np.zeros(obs.size)), obs.size, 1e-10, 1000, 0, p(z.copy()), p(z.copy()),
                                 p(z.copy()), ctypes.byref(J), its)
    assert rc == -1 and "observation" in L.host_poisson_error().decode()
    b = op.load(m, np.ones(m.n_nodes), w.mask)
    it, res = ctypes.c_int(), ctypes.c_double()
    rc = L.host_poisson_solve(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz, w.alpha, p(w.mask), p(b), p(np.zeros(m.n_nodes)),
                              1e-12, 5, 1, ctypes.byref(it), ctypes.byref(res))
    assert rc == -3 and it.value == 5 and "limit" in L.host_poisson_error().decode()


def test_edge_cases(L):
    """No observations (J = 0, zero gradient, zero adjoint iterations); a
    one-cell box whose every node is prescribed (u = b, no CG iteration);
    maxit = 0 on an unsolved system."""
    w = workload()
    m, _ = op.from_workload(w)
    n = m.n_nodes
    u, lam, g = np.zeros(n), np.ones(n), np.ones(n)
    J, its = ctypes.c_double(-1.0), (ctypes.c_int * 2)()
    empty = np.zeros(0, np.int64)
    rc = L.host_poisson_gradient(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz, w.alpha, p(w.mask), p(np.ones(n)), p(empty),
                                 p(np.zeros(0)), 0, 1e-10, 1000, 0, p(u), p(lam), p(g), ctypes.byref(J), its)
    assert rc == 0 and J.value == 0.0 and its[1] == 0 and np.all(lam == 0) and np.all(g == 0)
    mask1 = np.ones(8, np.uint8)
    b1 = np.arange(8, dtype=np.float64)
    u1 = np.zeros(8)
    it, res = ctypes.c_int(-1), ctypes.c_double(-1)
    for mixed in (0, 1):
        u1[:] = 0
        rc = L.host_poisson_solve(1, 1, 1, 1.0, 1.0, 1.0, 1.0, p(mask1), p(b1), p(u1), 1e-12, 100, mixed,
                                  ctypes.byref(it), ctypes.byref(res))
        assert rc == 0 and np.array_equal(u1, b1) and res.value <= 1e-12
    b = op.load(m, np.ones(n), w.mask)
    rc = L.host_poisson_solve(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz, w.alpha, p(w.mask), p(b), p(np.zeros(n)), 1e-10, 0,
                              0, ctypes.byref(it), ctypes.byref(res))
    assert rc == -3 and it.value == 0


def test_observation_on_a_prescribed_node(L):
    """An observed boundary node counts in J (u = 0 there) but feeds no
    adjoint load, as in the oracle (only free rows carry the adjoint)."""
    w = workload()
    m, prob = op.from_workload(w)
    obs = np.concatenate([w.obs[:5], np.flatnonzero(w.mask)[:3]]).astype(np.int64)
    rng = np.random.default_rng(12)
    theta = rng.standard_normal(m.n_nodes)
    u_obs = 0.01 * rng.standard_normal(obs.size)
    J_ref, g_ref, _, _ = prob.gradient(theta, obs, u_obs)
    u, lam, g = np.zeros(m.n_nodes), np.zeros(m.n_nodes), np.zeros(m.n_nodes)
    J, its = ctypes.c_double(), (ctypes.c_int * 2)()
    rc = L.host_poisson_gradient(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz, w.alpha, p(w.mask), p(theta), p(obs),
                                 p(u_obs), obs.size, 1e-12, 20000, 0, p(u), p(lam), p(g), ctypes.byref(J), its)
    assert rc == 0
    assert abs(J.value - J_ref) <= 1e-10 * J_ref
    assert np.linalg.norm(g - g_ref) <= 1e-8 * np.linalg.norm(g_ref)


def test_non_finite_input_is_reported(L):
    w = workload()
    m, _ = op.from_workload(w)
    b = op.load(m, np.ones(m.n_nodes), w.mask)
    b[int(np.flatnonzero(w.mask == 0)[3])] = np.nan
    it, res = ctypes.c_int(), ctypes.c_double()
    for mixed in (0, 1):
        rc = L.host_poisson_solve(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz, w.alpha, p(w.mask), p(b),
                                  p(np.zeros(m.n_nodes)), 1e-10, 100, mixed, ctypes.byref(it), ctypes.byref(res))
        assert rc == -6 and "non-finite" in L.host_poisson_error().decode()
