"""Property-based parity of the host builds of the CUDA library's
arithmetic against the oracle (hypothesis draws the cases): the Poisson
stencil rows on random boxes, lengths and masks, the J2 return map and its
tangent on random histories and strain increments, and the cone filter, its
transpose and the optimality-criteria step on random boxes, radii and
designs."""
import ctypes

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
from oracle import plasticity as pl, poisson as op  # noqa: E402
from tests import host_build  # noqa: E402

TAB = 27 * 27


def p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


_PC = None
_JC = None


def pcore():
    global _PC
    if _PC is None:
        _PC = host_build.build("poisson_core_host", extra_flags=["-ffp-contract=off"])
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        _PC.host_tables.argtypes = [D, D, D, D, P]
        _PC.host_apply.argtypes = [I, I, I, P, I, I, P, P, P]
    return _PC


def jcore():
    global _JC
    if _JC is None:
        _JC = host_build.build("j2_core_host", extra_flags=["-ffp-contract=off"])
        P, D = ctypes.c_void_p, ctypes.c_double
        _JC.host_j2_stress.argtypes = [D, D, D, P, P, P, P, P]
        _JC.host_j2_stress.restype = D
        _JC.host_j2_dstress.argtypes = [D, D, D, P, P, P, P, P]
    return _JC


@settings(max_examples=25, deadline=None, derandomize=True)
@given(nx=st.integers(1, 5), ny=st.integers(1, 5), nz=st.integers(1, 4),
       lx=st.floats(0.1, 3.0), ly=st.floats(0.1, 3.0), lz=st.floats(0.1, 3.0),
       alpha=st.floats(0.01, 100.0), density=st.floats(0.0, 1.0), seed=st.integers(0, 2 ** 31 - 1))
def test_poisson_stencil_rows(nx, ny, nz, lx, ly, lz, alpha, density, seed):
    L = pcore()
    m = oracle.mesh(nx, ny, nz, lx, ly, lz)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(m.n_nodes)
    mask = (rng.uniform(size=m.n_nodes) < density).astype(np.uint8)
    tab = np.zeros(2 * TAB)
    L.host_tables(lx / nx, ly / ny, lz / nz, alpha, p(tab))
    y = np.zeros(m.n_nodes)
    L.host_apply(nx, ny, nz, p(tab), 0, 0, p(x), p(mask), p(y))
    ref = op.apply(m, alpha, x, mask)
    assert np.abs(y - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    L.host_apply(nx, ny, nz, p(tab), 1, 1, p(x), p(mask), p(y))
    ref = op.load(m, x, mask)
    assert np.abs(y - ref).max() <= 1e-13 * max(1e-30, np.abs(ref).max()) + 1e-300


def six(T):
    return np.array([T[0, 0], T[1, 1], T[2, 2], T[1, 2], T[0, 2], T[0, 1]])


def full(s):
    return np.array([[s[0], s[5], s[4]], [s[5], s[1], s[3]], [s[4], s[3], s[2]]])


@settings(max_examples=60, deadline=None, derandomize=True)
@given(E=st.floats(1.0, 1e6), nu=st.floats(-0.5, 0.49), sy_frac=st.floats(1e-4, 1e-2),
       amp=st.floats(1e-6, 1e-1), seed=st.integers(0, 2 ** 31 - 1))
def test_j2_return_map_and_tangent(E, nu, sy_frac, amp, seed):
    L = jcore()
    sy = sy_frac * E
    mat = pl.Material(E, nu, sy)
    rng = np.random.default_rng(seed)
    e = rng.standard_normal((3, 3)) * sy_frac
    eo = 0.5 * (e + e.T)
    s = rng.standard_normal((3, 3)) * sy * 0.3
    so = 0.5 * (s + s.T)
    H = eo + rng.standard_normal((3, 3)) * amp
    dH = rng.standard_normal((3, 3))
    ref_sig, _, ref_f = pl.stress(mat, eo, so, H)
    sig, eps = np.zeros(6), np.zeros(6)
    f = L.host_j2_stress(E, nu, sy, p(six(eo)), p(six(so)), p(np.ascontiguousarray(H)), p(sig), p(eps))
    scale = max(sy, np.abs(ref_sig).max())
    assert abs(f - ref_f) <= 1e-10 * scale
    if abs(ref_f) <= 1e-9 * scale:
        return  # on the yield surface the branch is decided by rounding
    assert np.abs(full(sig) - ref_sig).max() <= 1e-10 * scale
    ds = np.zeros(6)
    L.host_j2_dstress(E, nu, sy, p(six(eo)), p(six(so)), p(np.ascontiguousarray(H)), p(np.ascontiguousarray(dH)),
                      p(ds))
    ref = pl.dstress(mat, eo, so, H, dH)
    assert np.abs(full(ds) - ref).max() <= 1e-9 * max(1e-300, np.abs(ref).max())


_TC = None


def tcore():
    global _TC
    if _TC is None:
        _TC = host_build.build("topopt_core_host", extra_flags=["-ffp-contract=off"])
        P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
        _TC.host_filter.argtypes = [P, P, I, I, I, D]
        _TC.host_filter_t.argtypes = [P, P, I, I, I, D]
        _TC.host_oc_step.argtypes = [I64, P, P, P, D, D, D, D, P]
        _TC.host_oc_step.restype = D
    return _TC


@settings(max_examples=30, deadline=None, derandomize=True)
@given(nx=st.integers(1, 7), ny=st.integers(1, 7), nz=st.integers(1, 4), rmin=st.floats(0.3, 4.0),
       seed=st.integers(0, 2 ** 31 - 1))
def test_filter_and_transpose(nx, ny, nz, rmin, seed):
    from oracle import topopt as ot
    L = tcore()
    g = np.random.default_rng(seed).standard_normal(nx * ny * nz)
    H = ot.filter_matrix(nx, ny, nz, rmin)
    out = np.zeros_like(g)
    L.host_filter(p(g), p(out), nx, ny, nz, rmin)
    assert np.abs(out - ot.filter_sensitivities(H, g)).max() <= 1e-13 * np.abs(g).max()
    L.host_filter_t(p(g), p(out), nx, ny, nz, rmin)
    assert np.abs(out - ot.filter_transpose(H, g)).max() <= 1e-13 * np.abs(g).max()


@settings(max_examples=30, deadline=None, derandomize=True)
@given(n=st.integers(1, 40), vol=st.floats(0.05, 0.95), move=st.floats(0.01, 0.5), seed=st.integers(0, 2 ** 31 - 1))
def test_oc_step(n, vol, move, seed):
    from oracle import topopt as ot
    L = tcore()
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.01, 1.0, n)
    g = -rng.uniform(0.0, 10.0, n) * (rng.uniform(size=n) < 0.9)
    dv = rng.uniform(0.5, 2.0, n)
    ref, lam_ref = ot.oc_step(x, g, dv, vol, move, 0.0, 1.0)
    y = np.zeros(n)
    lam = L.host_oc_step(n, p(x), p(np.ascontiguousarray(g)), p(dv), vol, move, 0.0, 1.0, p(y))
    assert np.abs(y - ref).max() <= 1e-12
