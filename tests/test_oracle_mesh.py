"""Pins of the oracle's integer subsystems: mesh, colouring, CSR, scatter map.

Closed forms: Ne = nx ny nz, N = (nx+1)(ny+1)(nz+1), nnz = 9 (3a-2)(3b-2)(3c-2)
with a = nx+1 ...; brute-force node-pair sets on tiny meshes; the colouring
invariant (no two cells of one colour share a node).
"""
import itertools

import numpy as np
import pytest

import oracle
from tests.indep import CORNERS

SIZES = [(1, 1, 1), (2, 2, 2), (3, 4, 5), (5, 2, 3)]


@pytest.mark.parametrize("n", SIZES)
def test_counts_closed_form(n):
    nx, ny, nz = n
    m = oracle.mesh(nx, ny, nz, 1.0, 2.0, 3.0)
    assert m.n_cells == nx * ny * nz
    assert m.n_nodes == (nx + 1) * (ny + 1) * (nz + 1)
    row_ptr, col = oracle.csr(m)
    a, b, c = nx + 1, ny + 1, nz + 1
    assert row_ptr[-1] == 9 * (3 * a - 2) * (3 * b - 2) * (3 * c - 2)
    assert len(col) == row_ptr[-1]


@pytest.mark.parametrize("n", SIZES)
def test_vtk_order_and_coords(n):
    nx, ny, nz = n
    lx, ly, lz = 1.0, 2.0, 3.0
    m = oracle.mesh(nx, ny, nz, lx, ly, lz)
    h = np.array([lx / nx, ly / ny, lz / nz])
    for e in range(m.n_cells):
        X = m.X[m.conn[e]]
        centre = X.mean(axis=0)
        # each local node sits at centre + sign * h/2 in VTK order
        assert np.allclose(X, centre + CORNERS * h / 2, atol=1e-12)
    assert np.allclose(m.X.min(axis=0), 0) and np.allclose(m.X.max(axis=0), [lx, ly, lz])
    # node numbering x fastest
    i, j, k = 1 % (nx + 1), 1 % (ny + 1), 1 % (nz + 1)
    node = i + (nx + 1) * (j + (ny + 1) * k)
    assert np.allclose(m.X[node], [i * h[0], j * h[1], k * h[2]])


@pytest.mark.parametrize("n", SIZES)
def test_csr_equals_brute_force_pairs(n):
    m = oracle.mesh(*n)
    pairs = set()
    for e in range(m.n_cells):
        for a, b in itertools.product(m.conn[e], m.conn[e]):
            for i in range(3):
                for j in range(3):
                    pairs.add((3 * int(a) + i, 3 * int(b) + j))
    row_ptr, col = oracle.csr(m)
    got = set()
    for r in range(m.n_dofs):
        cols = col[row_ptr[r]:row_ptr[r + 1]]
        assert np.all(np.diff(cols) > 0), "columns must be strictly ascending"
        got.update((r, int(cc)) for cc in cols)
    assert got == pairs


@pytest.mark.parametrize("n", SIZES)
def test_scatter_map(n):
    m = oracle.mesh(*n)
    row_ptr, col = oracle.csr(m)
    mp = oracle.scatter_map(m, row_ptr, col)
    for e in range(m.n_cells):
        for r in range(24):
            row = 3 * m.conn[e, r // 3] + r % 3
            for c in range(24):
                slot = mp[e, r, c]
                assert row_ptr[row] <= slot < row_ptr[row + 1]
                assert col[slot] == 3 * m.conn[e, c // 3] + c % 3


@pytest.mark.parametrize("n", SIZES + [(4, 4, 4)])
def test_colouring_invariant(n):
    nx, ny, nz = n
    m = oracle.mesh(nx, ny, nz)
    ptr, perm = oracle.colour(m)
    assert ptr[0] == 0 and ptr[8] == m.n_cells
    assert sorted(perm.tolist()) == list(range(m.n_cells))
    for c in range(8):
        cells = perm[ptr[c]:ptr[c + 1]]
        assert np.all(np.diff(cells) > 0), "stable (ascending) inside a colour"
        nodes = m.conn[cells].reshape(-1)
        assert len(np.unique(nodes)) == len(nodes), "no shared node within a colour"
        # colour formula
        i = cells % nx
        j = (cells // nx) % ny
        k = cells // (nx * ny)
        assert np.all((i & 1) + 2 * (j & 1) + 4 * (k & 1) == c)
