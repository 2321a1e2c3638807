"""CPU run of the library's J2 load step: the Newton control (j2_newton.h),
the CG control (dpcg_control.h) and the per-cell arithmetic (j2_core.cuh)
compiled for the host through tests/j2_step_host.cpp, with loops standing in
for the kernels; against the oracle's load-stepped Newton with direct solves
on the load / unload / reverse-yield path, and on a sheared box whose
yielding is not uniform."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import plasticity as pl
from paper_2212_00964_gb300 import inputs
from tests import host_build


@pytest.fixture(scope="module")
def L():
    lib = host_build.build("j2_step_host", extra_flags=[])
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.host_j2_step.argtypes = [I, I, I, D, D, D, D, D, D, P, P, P, P, D, I, D, I, I, ctypes.POINTER(I),
                                 ctypes.POINTER(I), ctypes.POINTER(ctypes.c_int64)]
    lib.host_j2_step_error.restype = ctypes.c_char_p
    return lib


def p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def six(T):
    return np.array([T[..., 0, 0], T[..., 1, 1], T[..., 2, 2], T[..., 1, 2], T[..., 0, 2], T[..., 0, 1]])


def to_soa(hist):
    eps, sig = hist
    return np.ascontiguousarray(np.concatenate([six(eps).transpose(0, 2, 1), six(sig).transpose(0, 2, 1)]).reshape(-1))


def run_path(L, dims, mat, mask, ubars, newton_maxit=30, mixed=False):
    nx, ny, nz, lx, ly, lz = dims
    D = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    u = np.zeros(D)
    hist = np.zeros(12 * 8 * nx * ny * nz)
    out = []
    for ub in ubars:
        ni, ci, nyd = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        rc = L.host_j2_step(nx, ny, nz, lx, ly, lz, mat.E, mat.nu, mat.sy, p(mask), p(np.ascontiguousarray(ub)),
                            p(u), p(hist), 1e-12, newton_maxit, 1e-4 if mixed else 1e-12, 20000, int(mixed),
                            ctypes.byref(ni), ctypes.byref(ci), ctypes.byref(nyd))
        out.append((rc, u.copy(), hist.copy(), ni.value, ci.value, nyd.value))
        if rc:
            break
    return out


@pytest.mark.parametrize("mixed", [False, True])
def test_uniaxial_path_matches_oracle(L, mixed):
    n = 3
    mask, ubars, strains, (E, nu, sy) = inputs.j2_uniaxial(n=n)
    mat = pl.Material(E, nu, sy)
    om = oracle.mesh(n, n, n)
    ref = pl.solve_path(om, mat, mask, ubars)
    got = run_path(L, (n, n, n, 1.0, 1.0, 1.0), mat, mask, ubars, mixed=mixed)
    for k, ((rc, u, h, ni, ci, nyd), (u_ref, hist_ref, ny_ref)) in enumerate(zip(got, ref)):
        assert rc == 0, (k, L.host_j2_step_error())
        assert np.abs(u - u_ref).max() <= 1e-10 * np.abs(u_ref).max()
        assert np.abs(h - to_soa(hist_ref)).max() <= 1e-8 * sy
        assert 1 <= ni <= (15 if mixed else 10)


def sheared_box():
    """2x3x2 box: bottom clamped, top pushed down and sheared; yielding
    spreads from the top corners (not uniform)."""
    nx, ny, nz = 2, 3, 2
    steps = [0.3e-2, 0.6e-2, 0.9e-2, 0.5e-2, 0.0]
    ubars = []
    mask = None
    for s in steps:
        mask, ub = inputs.dirichlet(nx, ny, nz, [("z0", 0, 0.0), ("z0", 1, 0.0), ("z0", 2, 0.0),
                                                 ("z1", 0, s), ("z1", 2, -0.5 * s)])
        ubars.append(ub)
    return (nx, ny, nz, 1.0, 1.5, 1.0), mask, ubars


@pytest.mark.parametrize("mixed", [False, True])
def test_sheared_box_matches_oracle(L, mixed):
    dims, mask, ubars = sheared_box()
    mat = pl.Material(70e3, 0.3, 250.0)
    om = oracle.mesh(*dims)
    ref = pl.solve_path(om, mat, mask, ubars)
    got = run_path(L, dims, mat, mask, ubars, mixed=mixed)
    mixes = 0
    for k, ((rc, u, h, ni, ci, nyd), (u_ref, hist_ref, ny_ref)) in enumerate(zip(got, ref)):
        assert rc == 0, (k, L.host_j2_step_error())
        assert np.abs(u - u_ref).max() <= 1e-9 * np.abs(u_ref).max()
        assert np.abs(h - to_soa(hist_ref)).max() <= 1e-7 * 250.0
        assert nyd == ny_ref
        mixes += 0 < ny_ref < 8 * om.n_cells
    assert mixes >= 1


def test_newton_limit_leaves_the_history(L):
    dims, mask, ubars = sheared_box()
    got = run_path(L, dims, pl.Material(70e3, 0.3, 250.0), mask, ubars[2:3], newton_maxit=0)
    rc, u, h, ni, ci, nyd = got[0]
    assert rc == -3 and "limit" in L.host_j2_step_error().decode() and np.all(h == 0)


def test_truncated_inner_solves_still_converge(L):
    """With at most 3 CG iterations per correction the step still reaches
    the oracle's solution: truncated inner solves are inexact Newton steps."""
    dims, mask, ubars = sheared_box()
    mat = pl.Material(70e3, 0.3, 250.0)
    nx, ny, nz, lx, ly, lz = dims
    D = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    u, hist = np.zeros(D), np.zeros(12 * 8 * nx * ny * nz)
    ni, ci, nyd = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    rc = L.host_j2_step(nx, ny, nz, lx, ly, lz, mat.E, mat.nu, mat.sy, p(mask), p(np.ascontiguousarray(ubars[0])),
                        p(u), p(hist), 1e-10, 200, 1e-12, 3, 0, ctypes.byref(ni), ctypes.byref(ci), ctypes.byref(nyd))
    assert rc == 0, L.host_j2_step_error()
    ref = pl.solve_path(oracle.mesh(*dims), mat, mask, ubars[:1])[0][0]
    assert np.abs(u - ref).max() <= 1e-8 * np.abs(ref).max()
    assert ni.value > 5


def test_edge_cases(L):
    """A one-cell box; a load step that changes nothing (converged at
    iteration 0, history kept); a step back to the virgin state."""
    mat = pl.Material(70e3, 0.3, 250.0)
    mask, ubars, strains, _ = inputs.j2_uniaxial(n=1)
    got = run_path(L, (1, 1, 1, 1.0, 1.0, 1.0), mat, mask, ubars[:4])
    ref = pl.solve_path(oracle.mesh(1, 1, 1), mat, mask, ubars[:4])
    for (rc, u, h, ni, ci, nyd), (u_ref, hist_ref, ny_ref) in zip(got, ref):
        assert rc == 0 and np.abs(u - u_ref).max() <= 1e-10 * np.abs(u_ref).max()
    # repeating the last prescribed state: nothing to do
    rc, u, h, ni, ci, nyd = got[-1]
    again = run_path(L, (1, 1, 1, 1.0, 1.0, 1.0), mat, mask, [ubars[3]] * 1)
    assert again[0][0] == 0
    D = 3 * 8
    uu, hh = u.copy(), h.copy()
    ni2, ci2, ny2 = ctypes.c_int(-1), ctypes.c_int(-1), ctypes.c_int64(-1)
    rc = L.host_j2_step(1, 1, 1, 1.0, 1.0, 1.0, mat.E, mat.nu, mat.sy, p(mask), p(np.ascontiguousarray(ubars[3])),
                        p(uu), p(hh), 1e-12, 30, 1e-12, 1000, 0, ctypes.byref(ni2), ctypes.byref(ci2),
                        ctypes.byref(ny2))
    assert rc == 0 and ni2.value == 0 and ci2.value == 0
    assert np.array_equal(uu, u) and np.abs(hh - h).max() <= 1e-12 * np.abs(h).max()
    assert uu.size == D


@pytest.mark.parametrize("mixed", [False, True])
def test_one_large_step_far_into_plastic_flow(L, mixed):
    """A single step to a 10% shear and compression of the sheared box:
    Newton with the consistent tangent reaches the oracle's solution in a
    few iterations, in FP64 and with FP32 inner solves."""
    nx, ny, nz = 2, 3, 2
    s = 0.1
    mask, ub = inputs.dirichlet(nx, ny, nz, [("z0", 0, 0.0), ("z0", 1, 0.0), ("z0", 2, 0.0), ("z1", 0, s),
                                             ("z1", 2, -0.5 * s)])
    dims = (nx, ny, nz, 1.0, 1.5, 1.0)
    mat = pl.Material(70e3, 0.3, 250.0)
    ref = pl.solve_path(oracle.mesh(*dims), mat, mask, [ub])[0][0]
    rc, u, h, ni, ci, nyd = run_path(L, dims, mat, mask, [ub], newton_maxit=50, mixed=mixed)[0]
    assert rc == 0 and ni <= 12
    assert np.abs(u - ref).max() <= 1e-10 * np.abs(ref).max()


def random_paths(seed, n):
    """Random boxes clamped at z=0 with a random 4-step displacement path of
    the z=1 face."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx, ny, nz = rng.integers(1, 4, 3)
        dims = (int(nx), int(ny), int(nz), float(rng.uniform(0.5, 2)), float(rng.uniform(0.5, 2)),
                float(rng.uniform(0.5, 2)))
        path = np.cumsum(rng.standard_normal((4, 3)) * 4e-3, axis=0)
        ubars = []
        mask = None
        for d in path:
            mask, ub = inputs.dirichlet(dims[0], dims[1], dims[2], [("z0", 0, 0.0), ("z0", 1, 0.0), ("z0", 2, 0.0),
                                                                ("z1", 0, d[0]), ("z1", 1, d[1]), ("z1", 2, d[2])])
            ubars.append(ub)
        out.append((dims, mask, ubars))
    return out


@pytest.mark.parametrize("mixed", [False, True])
def test_random_load_paths_match_the_oracle(L, mixed):
    """Random non-proportional paths (seed 5, the first six; the fifth once
    diverged before truncated CG and backtracking): wherever the oracle's
    exact Newton converges, the library reaches the same solution."""
    mat = pl.Material(70e3, 0.3, 250.0)
    compared = 0
    for dims, mask, ubars in random_paths(5, 6):
        try:
            ref = pl.solve_path(oracle.mesh(*dims), mat, mask, ubars)
        except (RuntimeError, pl.np.linalg.LinAlgError):
            continue
        got = run_path(L, dims, mat, mask, ubars, newton_maxit=50, mixed=mixed)
        for (rc, u, h, ni, ci, nyd), (u_ref, _, _) in zip(got, ref):
            assert rc == 0, L.host_j2_step_error()
            assert np.abs(u - u_ref).max() <= 1e-8 * np.abs(u_ref).max()
        compared += 1
    assert compared >= 4


def test_non_finite_prescribed_value_is_reported(L):
    dims, mask, ubars = sheared_box()
    ub = np.array(ubars[0])
    ub[np.flatnonzero(mask)[-1]] = np.nan
    got = run_path(L, dims, pl.Material(70e3, 0.3, 250.0), mask, [ub])
    assert got[0][0] == -6 and "non-finite" in L.host_j2_step_error().decode()
