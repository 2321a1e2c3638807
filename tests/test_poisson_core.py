"""CPU checks of the CUDA library's Poisson stencil arithmetic
(csrc/poisson_core.cuh, host/device functions compiled here with g++ through
tests/poisson_core_host.cpp) against the oracle's assembled operators: the
27-class stencil tables and the row formula, and the separable (tensor-
product) form the GPU kernel evaluates, index arithmetic included, on
anisotropic boxes, one-cell-thick boxes and arbitrary masks."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import poisson as op
from paper_2212_00964_gb300 import inputs
from tests import host_build

TAB = 27 * 27
OUT_ELIM, OUT_ZERO, OUT_PLAIN = 0, 1, 2


@pytest.fixture(scope="module")
def core():
    L = host_build.build("poisson_core_host", extra_flags=['-ffp-contract=off'])
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.host_tables.argtypes = [D, D, D, D, P]
    L.host_apply.argtypes = [I, I, I, P, I, I, P, P, P]
    L.host_apply_f32.argtypes = [I, I, I, P, I, I, P, P, P]
    L.host_diag.argtypes = [I, I, I, P, P, P]
    L.host_apply_sep.argtypes = [I, I, I, D, D, D, D, I, I, P, P, P]
    L.host_diag_sep.argtypes = [I, I, I, D, D, D, D, P, P]
    return L


def p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def tables(L, nx, ny, nz, lx, ly, lz, alpha):
    tab = np.zeros(2 * TAB)
    L.host_tables(lx / nx, ly / ny, lz / nz, alpha, p(tab))
    return tab


def apply(L, dims, tab, opi, mode, x, mask, f32=False):
    nx, ny, nz = dims
    if f32:
        x = np.ascontiguousarray(x, np.float32)
        y = np.zeros_like(x)
        L.host_apply_f32(nx, ny, nz, p(tab), opi, mode, p(x), p(mask), p(y))
    else:
        x = np.ascontiguousarray(x, np.float64)
        y = np.zeros_like(x)
        L.host_apply(nx, ny, nz, p(tab), opi, mode, p(x), p(mask), p(y))
    return y


CASES = [(3, 4, 2, 1.0, 1.3, 0.4), (1, 2, 1, 0.5, 1.0, 0.2), (5, 1, 3, 2.0, 0.3, 0.9), (1, 1, 1, 1.0, 1.0, 1.0)]


@pytest.mark.parametrize("case", CASES)
def test_tables_match_oracle_assembly(core, case):
    """Plain products (no mask) of both tables = the oracle's assembled A
    and M applied to a random vector."""
    nx, ny, nz, lx, ly, lz = case
    alpha = 1.7
    m = oracle.mesh(nx, ny, nz, lx, ly, lz)
    A, M = op.assemble(m, alpha)
    tab = tables(core, nx, ny, nz, lx, ly, lz, alpha)
    x = np.random.default_rng(1).standard_normal(m.n_nodes)
    yA = apply(core, (nx, ny, nz), tab, 0, OUT_PLAIN, x, None)
    yM = apply(core, (nx, ny, nz), tab, 1, OUT_PLAIN, x, None)
    assert np.abs(yA - A @ x).max() <= 1e-13 * np.abs(A @ x).max()
    assert np.abs(yM - M @ x).max() <= 1e-13 * np.abs(M @ x).max()


@pytest.mark.parametrize("case", CASES)
def test_masked_modes_match_oracle(core, case):
    """The eliminated stiffness (y_c = x_c) and the masked load (F_c = 0)
    with a random mask = the oracle's matrix-free apply and load; the
    Jacobi diagonal = the diagonal of the eliminated assembled matrix."""
    nx, ny, nz, lx, ly, lz = case
    alpha = 0.8
    m = oracle.mesh(nx, ny, nz, lx, ly, lz)
    rng = np.random.default_rng(2)
    mask = (rng.uniform(size=m.n_nodes) < 0.3).astype(np.uint8)
    tab = tables(core, nx, ny, nz, lx, ly, lz, alpha)
    x = rng.standard_normal(m.n_nodes)
    y = apply(core, (nx, ny, nz), tab, 0, OUT_ELIM, x, mask)
    ref = op.apply(m, alpha, x, mask)
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
    F = apply(core, (nx, ny, nz), tab, 1, OUT_ZERO, x, mask)
    refF = op.load(m, x, mask)
    assert np.abs(F - refF).max() <= 1e-13 * np.abs(refF).max()
    d = np.zeros(m.n_nodes)
    core.host_diag(nx, ny, nz, p(tab), p(mask), p(d))
    A, _ = op.assemble(m, alpha)
    dref = np.where(mask == 1, 1.0, A.diagonal())
    assert np.abs(d - dref).max() <= 1e-13 * np.abs(dref).max()


def test_fp32_rows(core):
    """The float instantiation agrees with the oracle to float rounding."""
    nx, ny, nz = 6, 5, 4
    m = oracle.mesh(nx, ny, nz, 1.0, 1.0, 0.2)
    mask = inputs.boundary_nodes(nx, ny, nz)
    tab = tables(core, nx, ny, nz, 1.0, 1.0, 0.2, 1.0)
    x = np.random.default_rng(3).standard_normal(m.n_nodes)
    y = apply(core, (nx, ny, nz), tab, 0, OUT_ELIM, x, mask, f32=True)
    ref = op.apply(m, 1.0, x, mask)
    assert np.abs(y - ref).max() <= 2e-6 * np.abs(ref).max()


def test_table_invariants(core):
    """Every stiffness class sums to 0 (constants carry no gradient); the
    mass classes sum to the volume of the cells around the node (8 cells
    inside, 1 at a corner) divided by 8 per cell."""
    h = (0.3, 0.5, 0.7)
    tab = np.zeros(2 * TAB)
    core.host_tables(*h, 2.0, p(tab))
    K = tab[:TAB].reshape(27, 27)
    M = tab[TAB:].reshape(27, 27)
    assert np.abs(K.sum(axis=1)).max() <= 1e-14 * np.abs(K).max()
    V = np.prod(h)
    for cls in range(27):
        c = [cls % 3, (cls // 3) % 3, cls // 9]
        n_cells = np.prod([2 if ci == 1 else 1 for ci in c])
        assert abs(M[cls].sum() - n_cells * V / 8) <= 1e-15


def apply_sep(L, case, alpha, opi, mode, x, mask):
    nx, ny, nz, lx, ly, lz = case
    x = np.ascontiguousarray(x, np.float64)
    y = np.zeros_like(x)
    L.host_apply_sep(nx, ny, nz, lx, ly, lz, alpha, opi, mode, p(x), p(mask), p(y))
    return y


@pytest.mark.parametrize("case", CASES)
def test_separable_rows_match_oracle(core, case):
    """The separable rows (per-axis 1D stiffness and mass stencils combined
    as alpha (Kx My Mz + Mx Ky Mz + Mx My Kz) and Mx My Mz) = the oracle's
    assembled A and M, plain and with a random mask in both masked modes; the
    separable Jacobi diagonal = the eliminated assembled diagonal."""
    nx, ny, nz, lx, ly, lz = case
    alpha = 1.3
    m = oracle.mesh(nx, ny, nz, lx, ly, lz)
    A, M = op.assemble(m, alpha)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(m.n_nodes)
    mask = (rng.uniform(size=m.n_nodes) < 0.3).astype(np.uint8)
    yA = apply_sep(core, case, alpha, 0, OUT_PLAIN, x, None)
    yM = apply_sep(core, case, alpha, 1, OUT_PLAIN, x, None)
    assert np.abs(yA - A @ x).max() <= 1e-13 * np.abs(A @ x).max()
    assert np.abs(yM - M @ x).max() <= 1e-13 * np.abs(M @ x).max()
    y = apply_sep(core, case, alpha, 0, OUT_ELIM, x, mask)
    ref = op.apply(m, alpha, x, mask)
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()
    F = apply_sep(core, case, alpha, 1, OUT_ZERO, x, mask)
    refF = op.load(m, x, mask)
    assert np.abs(F - refF).max() <= 1e-13 * np.abs(refF).max()
    d = np.zeros(m.n_nodes)
    core.host_diag_sep(nx, ny, nz, lx, ly, lz, alpha, p(mask), p(d))
    dref = np.where(mask == 1, 1.0, A.diagonal())
    assert np.abs(d - dref).max() <= 1e-13 * np.abs(dref).max()
