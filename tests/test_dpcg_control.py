"""CPU checks of the host control of the device-scalar Jacobi-PCG
(csrc/dpcg_control.h) that the Poisson and J2 paths share, driven through
tests/dpcg_control_host.cpp by CPU stand-ins of its kernels: convergence to
numpy's solution, the batching of iterations between host reads, and the
exits (already converged, zero right-hand side, iteration limit, negative
curvature in the first iteration (breakdown) or later (truncation at the
last iterate), non-finite input)."""
import ctypes

import numpy as np
import pytest

from tests import host_build

OK, NOT_CONVERGED, BREAKDOWN, NONFINITE = 0, -3, -5, -6
CHECK = 8


@pytest.fixture(scope="module")
def L():
    lib = host_build.build("dpcg_control_host", extra_flags=[])
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.host_pcg.argtypes = [I, P, P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(I)]
    lib.host_pcg_error.restype = ctypes.c_char_p
    return lib


def p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def run(L, A, b, u0=None, rtol=1e-12, maxit=500):
    A = np.ascontiguousarray(A, np.float64)
    n = A.shape[0]
    d = np.diag(A)
    dinv = np.where(d != 0, 1.0 / np.where(d != 0, d, 1.0), 0.0)
    u = np.zeros(n) if u0 is None else np.array(u0, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    it, res, calls = ctypes.c_int(-1), ctypes.c_double(-1), ctypes.c_int(-1)
    rc = L.host_pcg(n, p(A), p(dinv), p(b), p(u), rtol, maxit, ctypes.byref(it), ctypes.byref(res),
                    ctypes.byref(calls))
    return rc, u, it.value, res.value, calls.value, L.host_pcg_error().decode()


def spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return Q @ np.diag(np.geomspace(1.0, cond, n)) @ Q.T


def test_converges_to_the_solution(L):
    A = spd(60, 1)
    b = np.random.default_rng(2).standard_normal(60)
    rc, u, it, res, calls, _ = run(L, A, b)
    assert rc == OK
    assert np.linalg.norm(A @ u - b) <= 1e-11 * np.linalg.norm(b)
    # the reported residual is CG's recursively updated one (the true one
    # stagnates at the rounding level, which the line above bounds)
    assert res <= 1e-12
    assert it % CHECK == 0 and calls == it // CHECK


def test_exact_start_and_zero_rhs(L):
    A = spd(20, 3)
    b = np.random.default_rng(4).standard_normal(20)
    rc, u, it, res, _, _ = run(L, A, b, u0=np.linalg.solve(A, b), rtol=1e-8)
    assert rc == OK and it == 0
    rc, u, it, res, _, _ = run(L, A, np.zeros(20))
    assert rc == OK and it == 0 and res == 0.0 and np.all(u == 0)


def test_iteration_limit(L):
    A = spd(80, 5, cond=1e8)
    b = np.random.default_rng(6).standard_normal(80)
    rc, u, it, res, calls, err = run(L, A, b, maxit=11)
    assert rc == NOT_CONVERGED and it == 11 and calls == 2 and "limit" in err and res > 1e-12


def test_negative_curvature_first_is_a_breakdown(L):
    A = -spd(12, 10)
    rc, _, it, _, _, err = run(L, A, np.ones(12))
    assert rc == BREAKDOWN and "positive definite" in err


def test_negative_curvature_later_truncates_at_the_last_iterate(L):
    """An indefinite operator whose first directions have positive
    curvature: the solve stops at the iterate reached before the first
    p^T A p <= 0 (the later iterations of the batch change nothing), and the
    reported residual is that iterate's."""
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    A = Q @ np.diag(np.linspace(-1.0, 2.0, 30)) @ Q.T
    b = rng.standard_normal(30)
    rc, u, it, res, _, err = run(L, A, b, maxit=200)
    assert rc == NOT_CONVERGED and "truncated" in err
    assert np.all(np.isfinite(u)) and np.any(u != 0)
    assert abs(np.linalg.norm(b - A @ u) / np.linalg.norm(b) - res) <= 1e-8


def test_non_finite_input(L):
    A = spd(10, 8)
    b = np.ones(10)
    b[3] = np.nan
    rc, _, it, _, _, err = run(L, A, b)
    assert rc == NONFINITE and "non-finite" in err


def test_zero_iteration_limit(L):
    A = spd(10, 9)
    rc, u, it, res, calls, err = run(L, A, np.ones(10), maxit=0)
    assert rc == NOT_CONVERGED and it == 0 and calls == 0 and np.all(u == 0)
    rc, u, it, res, calls, err = run(L, A, np.zeros(10), maxit=0)
    assert rc == OK and it == 0


def test_reported_residual_is_the_final_one(L):
    """Away from the rounding floor CG's recursive residual equals the true
    one, so the reported ||r|| / ||b|| must match ||b - A u|| / ||b|| of the
    returned iterate (the last of its batch)."""
    A = spd(40, 11, cond=1e2)
    b = np.random.default_rng(12).standard_normal(40)
    rc, u, it, res, calls, _ = run(L, A, b, rtol=1e-6)
    true = np.linalg.norm(b - A @ u) / np.linalg.norm(b)
    assert rc == OK and res <= 1e-6
    assert abs(res - true) <= 1e-9
