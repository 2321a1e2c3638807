"""CPU checks of the CUDA library's J2 plasticity arithmetic
(csrc/j2_core.cuh, host/device functions compiled here with g++ through
tests/j2_core_host.cpp): the return map and its tangent per Gauss point,
and the per-cell residual and tangent assembled over a box, against the
oracle (Sec. 2.3, Eqs. (14)-(15)), with the history in the kernels'
structure-of-arrays layout."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import plasticity as pl
from paper_2212_00964_gb300 import inputs
from tests import host_build

MAT = pl.Material(70e3, 0.3, 250.0)


@pytest.fixture(scope="module")
def core():
    L = host_build.build("j2_core_host", extra_flags=['-ffp-contract=off'])
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    L.host_j2_stress.argtypes = [D, D, D, P, P, P, P, P]
    L.host_j2_stress.restype = D
    L.host_j2_dstress.argtypes = [D, D, D, P, P, P, P, P]
    L.host_j2_residual.argtypes = [I, I, I, D, D, D, D, D, D, P, P, P, P, P]
    L.host_j2_residual.restype = I64
    L.host_j2_apply.argtypes = [I, I, I, D, D, D, D, D, D, P, P, P, P, P]
    L.host_j2_diag.argtypes = [I, I, I, D, D, D, D, D, D, P, P, P, I]
    return L


def p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def six(T):
    """3x3 symmetric -> (xx, yy, zz, yz, xz, xy)."""
    T = np.asarray(T)
    return np.array([T[..., 0, 0], T[..., 1, 1], T[..., 2, 2], T[..., 1, 2], T[..., 0, 2], T[..., 0, 1]])


def full(s):
    return np.array([[s[0], s[5], s[4]], [s[5], s[1], s[3]], [s[4], s[3], s[2]]])


def to_soa(hist):
    """oracle history ([Ne, 8, 3, 3] eps, sigma) -> hist[(comp*8 + q)*Ne + e]."""
    eps, sig = hist
    ne = eps.shape[0]
    out = np.zeros((12, 8, ne))
    out[:6] = six(eps).transpose(0, 2, 1)
    out[6:] = six(sig).transpose(0, 2, 1)
    return np.ascontiguousarray(out.reshape(-1))


def from_soa(h, ne):
    h = h.reshape(12, 8, ne)
    eps = np.zeros((ne, 8, 3, 3))
    sig = np.zeros((ne, 8, 3, 3))
    for e in range(ne):
        for q in range(8):
            eps[e, q] = full(h[:6, q, e])
            sig[e, q] = full(h[6:, q, e])
    return eps, sig


def test_point_stress_and_tangent(core):
    rng = np.random.default_rng(1)
    n_pl = 0
    for _ in range(60):
        e = rng.standard_normal((3, 3)) * 2e-3
        eo = 0.5 * (e + e.T)
        s = rng.standard_normal((3, 3)) * 80
        so = 0.5 * (s + s.T)
        H = eo + rng.standard_normal((3, 3)) * 4e-3
        dH = rng.standard_normal((3, 3))
        ref_sig, ref_eps, ref_f = pl.stress(MAT, eo, so, H)
        sig = np.zeros(6)
        eps = np.zeros(6)
        f = core.host_j2_stress(MAT.E, MAT.nu, MAT.sy, p(six(eo).copy()), p(six(so).copy()),
                                p(np.ascontiguousarray(H)), p(sig), p(eps))
        n_pl += f > 0
        assert abs(f - ref_f) <= 1e-10 * MAT.sy
        assert np.abs(full(sig) - ref_sig).max() <= 1e-10 * MAT.sy
        assert np.abs(full(eps) - ref_eps).max() <= 1e-16
        ds = np.zeros(6)
        core.host_j2_dstress(MAT.E, MAT.nu, MAT.sy, p(six(eo).copy()), p(six(so).copy()), p(np.ascontiguousarray(H)),
                             p(np.ascontiguousarray(dH)), p(ds))
        ref = pl.dstress(MAT, eo, so, H, dH)
        assert np.abs(full(ds) - ref).max() <= 1e-10 * np.abs(ref).max()
    assert 10 < n_pl < 60


def random_history(m, rng, scale_e=2e-3):
    """A plastically admissible history: one oracle residual pass from zero."""
    u = scale_e * rng.standard_normal(m.n_dofs)
    _, hist, _ = pl.residual(m, MAT, pl.zero_history(m), u)
    return hist, u


@pytest.mark.parametrize("dims", [(2, 3, 2, 1.0, 1.2, 0.8), (1, 1, 3, 0.5, 0.5, 1.5)])
def test_cell_residual_and_tangent_over_a_box(core, dims):
    nx, ny, nz, lx, ly, lz = dims
    m = oracle.mesh(nx, ny, nz, lx, ly, lz)
    rng = np.random.default_rng(nx * 7 + nz)
    hist, u1 = random_history(m, rng)
    u = u1 + 1e-3 * rng.standard_normal(m.n_dofs)
    mask = np.zeros(m.n_dofs, np.uint8)
    mask[3 * inputs.face_nodes(nx, ny, nz, "z0")] = 1
    mask[3 * inputs.face_nodes(nx, ny, nz, "z0") + 2] = 1
    R_ref, (eps_ref, sig_ref), ny_ref = pl.residual(m, MAT, hist, u, mask)
    h = to_soa(hist)
    R = np.zeros(m.n_dofs)
    h_new = np.zeros_like(h)
    n_y = core.host_j2_residual(nx, ny, nz, lx, ly, lz, MAT.E, MAT.nu, MAT.sy, p(u), p(h), p(mask), p(R), p(h_new))
    assert n_y == ny_ref and 0 < n_y < 8 * m.n_cells
    assert np.abs(R - R_ref).max() <= 1e-10 * np.abs(R_ref).max()
    e2, s2 = from_soa(h_new, m.n_cells)
    assert np.abs(s2 - sig_ref).max() <= 1e-10 * MAT.sy
    assert np.abs(e2 - eps_ref).max() <= 1e-15
    x = rng.standard_normal(m.n_dofs)
    y = np.zeros(m.n_dofs)
    core.host_j2_apply(nx, ny, nz, lx, ly, lz, MAT.E, MAT.nu, MAT.sy, p(u), p(h), p(x), p(mask), p(y))
    y_ref = pl.tangent_apply(m, MAT, hist, u, x, mask)
    assert np.abs(y - y_ref).max() <= 1e-10 * np.abs(y_ref).max()


@pytest.mark.parametrize("fp32", [0, 1])
def test_cell_diagonal_equals_the_assembled_diagonal(core, fp32):
    """The closed-form element diagonal (nine tangent directions per Gauss
    point) summed over a box = the diagonal of the oracle's assembled
    tangent, on a partly yielded state; in FP32 to float rounding."""
    nx, ny, nz, lx, ly, lz = 3, 2, 2, 1.2, 0.8, 0.6
    m = oracle.mesh(nx, ny, nz, lx, ly, lz)
    rng = np.random.default_rng(31)
    hist, u1 = random_history(m, rng, 6e-4)
    u = u1 + 3e-4 * rng.standard_normal(m.n_dofs)
    _, _, n_y = pl.residual(m, MAT, hist, u)
    assert 0 < n_y < 8 * m.n_cells
    d = np.zeros(m.n_dofs)
    core.host_j2_diag(nx, ny, nz, lx, ly, lz, MAT.E, MAT.nu, MAT.sy, p(u), p(to_soa(hist)), p(d), fp32)
    ref = pl.assemble(m, MAT, hist, u).diagonal()
    assert np.abs(d - ref).max() <= (2e-6 if fp32 else 1e-12) * np.abs(ref).max()
