"""The all-cores oracle operators (CPU baseline only) equal the serial ones:
same per-cell arithmetic, colour-class parallel scatter, so the results
differ only in the order of the additions into each node."""
import numpy as np
import pytest

import oracle
from paper_2212_00964_gb300 import inputs


@pytest.mark.parametrize("kind", [oracle.LINEAR, oracle.SIMP, oracle.NEOHOOKE])
def test_mt_operators_match_serial(kind):
    nx, ny, nz = 7, 5, 6
    m = oracle.mesh(nx, ny, nz, 1.0, 0.8, 1.2)
    mat = oracle.Material(kind, 10.0, 0.3)
    rng = np.random.default_rng(3)
    u = inputs.random_state(m.n_dofs, 0.15, 4, scale=0.05)
    x = inputs.random_vector(m.n_dofs, 5)
    f = inputs.random_vector(m.n_dofs, 6)
    cp = rng.uniform(0.1, 1.0, m.n_cells)
    mask, _ = inputs.clamp_and_compress(nx, ny, nz, -0.1)
    y = oracle.tangent_apply(m, mat, u, x, cp, mask)
    y_mt = oracle.tangent_apply_mt(m, mat, u, x, cp, mask)
    assert np.abs(y_mt - y).max() <= 1e-13 * np.abs(y).max()
    R = oracle.residual(m, mat, u, cp, f, mask)
    R_mt = oracle.residual_mt(m, mat, u, cp, f, mask)
    assert np.abs(R_mt - R).max() <= 1e-13 * np.abs(R).max()
    assert oracle.threads() >= 1
