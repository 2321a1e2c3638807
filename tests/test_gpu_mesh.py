"""GPU parity of the integer subsystems (bit-exact): connectivity,
coordinates, colouring, CSR pattern and scatter map, against the oracle."""
import numpy as np
import pytest

import oracle
from tests.gpu_common import fem, host

pytestmark = pytest.mark.gpu

SIZES = [(1, 1, 1), (2, 2, 2), (3, 4, 5), (8, 8, 8), (17, 9, 5)]


@pytest.mark.parametrize("n", SIZES)
def test_mesh_bit_exact(n):
    F = fem()
    lx, ly, lz = 1.0, 0.7, 1.3
    m = F.fem_mesh(*n, lx, ly, lz, csr=True)
    out = F.fem_mesh_export(m, csr=True)
    om = oracle.mesh(*n, lx, ly, lz)
    assert np.array_equal(host(out["conn"]), om.conn)
    assert np.array_equal(host(out["X"]), om.X)  # same IEEE formula -> identical bits
    ptr, perm = oracle.colour(om)
    assert np.array_equal(host(out["colour_ptr"]), ptr)
    assert np.array_equal(host(out["cell_perm"]), perm)
    rp, col = oracle.csr(om)
    assert m.nnz == rp[-1]
    assert np.array_equal(host(out["row_ptr"]).astype(np.int64), rp)
    assert np.array_equal(host(out["col"]), col)
    assert np.array_equal(host(out["map"]), oracle.scatter_map(om, rp, col))


def test_mesh_full_size_closed_forms_and_sampled_rows():
    """64^3 (the Neo-Hookean benchmark mesh): counts by closed form, sampled
    CSR rows by brute force over the cells around each node."""
    F = fem()
    n = 64
    m = F.fem_mesh(n, n, n, csr=True)
    a = n + 1
    assert m.n_nodes == a ** 3 and m.n_cells == n ** 3
    assert m.nnz == 9 * (3 * a - 2) ** 3
    out = F.fem_mesh_export(m, csr=True)
    rp = host(out["row_ptr"]).astype(np.int64)
    col = host(out["col"])
    conn = host(out["conn"])
    assert rp[-1] == m.nnz and np.all(np.diff(rp) > 0)
    rng = np.random.default_rng(0)
    for node in list(rng.integers(0, m.n_nodes, 40)) + [0, m.n_nodes - 1]:
        I, J, K = node % a, (node // a) % a, node // (a * a)
        cells = [ci + n * (cj + n * ck) for ck in (K - 1, K) for cj in (J - 1, J) for ci in (I - 1, I)
                 if 0 <= ci < n and 0 <= cj < n and 0 <= ck < n]
        nb = np.unique(conn[cells].reshape(-1))
        expect = (3 * nb[:, None] + np.arange(3)).reshape(-1)
        for c in range(3):
            r = 3 * node + c
            assert np.array_equal(col[rp[r]:rp[r + 1]], expect)
    ptr = host(out["colour_ptr"])
    perm = host(out["cell_perm"])
    assert ptr[-1] == m.n_cells and np.array_equal(np.sort(perm), np.arange(m.n_cells))
