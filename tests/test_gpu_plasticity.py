"""GPU parity of perfect J2 plasticity (Sec. 2.3, Eqs. (14)-(15)): the
residual with its returned history, the consistent tangent, and load-stepped
Newton (fem_j2_step) over the load / unload / reverse-yield path, against the
oracle and against the uniaxial closed form."""
import numpy as np
import pytest
import torch

import oracle
from oracle import plasticity as pl
from paper_2212_00964_gb300 import inputs
from tests.gpu_common import dev, fem, host, rel_l2

pytestmark = pytest.mark.gpu

E, NU, SY = 70e3, 0.3, 250.0


def six(T):
    return np.array([T[..., 0, 0], T[..., 1, 1], T[..., 2, 2], T[..., 1, 2], T[..., 0, 2], T[..., 0, 1]])


def to_soa(hist):
    eps, sig = hist
    out = np.concatenate([six(eps).transpose(0, 2, 1), six(sig).transpose(0, 2, 1)])
    return np.ascontiguousarray(out.reshape(-1))


def test_residual_and_tangent_parity():
    nx, ny, nz = 5, 3, 4
    F = fem()
    m = F.fem_mesh(nx, ny, nz, 1.0, 0.6, 0.8)
    om = oracle.mesh(nx, ny, nz, 1.0, 0.6, 0.8)
    omat = pl.Material(E, NU, SY)
    rng = np.random.default_rng(3)
    # amplitudes giving a mix: 396 of 480 points yield in the first state, 325 in the second
    u1 = 5e-4 * rng.standard_normal(om.n_dofs)
    _, hist, _ = pl.residual(om, omat, pl.zero_history(om), u1)
    u = u1 + 2e-4 * rng.standard_normal(om.n_dofs)
    mask = np.zeros(om.n_dofs, np.uint8)
    mask[3 * inputs.face_nodes(nx, ny, nz, "x0")] = 1
    R_ref, new_ref, ny_ref = pl.residual(om, omat, hist, u, mask)
    mat = F.j2_material(E, NU, SY)
    h_new = torch.zeros(12 * 8 * om.n_cells, dtype=torch.float64, device="cuda")
    r, n_y = F.fem_j2_residual(m, mat, dev(u), dev(to_soa(hist)), dev(mask), hist_new=h_new)
    assert n_y == ny_ref and 0 < n_y < 8 * om.n_cells
    assert rel_l2(host(r), R_ref) <= 1e-10
    assert rel_l2(host(h_new), to_soa(new_ref)) <= 1e-12
    x = rng.standard_normal(om.n_dofs)
    ref = pl.tangent_apply(om, omat, hist, u, x, mask)
    y = F.fem_j2_tangent_apply(m, mat, dev(u), dev(to_soa(hist)), dev(x), dev(mask))
    assert rel_l2(host(y), ref) <= 1e-10
    y32 = F.fem_j2_tangent_apply(m, mat, dev(u), dev(to_soa(hist)), dev(x, torch.float32), dev(mask))
    assert y32.dtype == torch.float32 and rel_l2(host(y32), ref) <= 1e-5


@pytest.mark.parametrize("mixed", [False, True])
def test_load_unload_path_vs_oracle_and_closed_form(mixed):
    n, L = 4, 1.0
    mask, ubars, strains, (E_, nu, sy) = inputs.j2_uniaxial(n=n, L=L)
    F = fem()
    m = F.fem_mesh(n, n, n, L, L, L)
    om = oracle.mesh(n, n, n, L, L, L)
    ref_path = pl.solve_path(om, pl.Material(E_, nu, sy), mask, ubars)
    mat = F.j2_material(E_, nu, sy)
    u = torch.zeros(om.n_dofs, dtype=torch.float64, device="cuda")
    hist = F.j2_history(m)
    mask_d = dev(mask)
    sig_prev, e_prev = 0.0, 0.0
    for k, ub in enumerate(ubars):
        st = F.fem_j2_step(m, mat, mask_d, dev(ub), u, hist, newton_rtol=1e-12, cg_rtol=1e-4 if mixed else 1e-12,
                           mixed=mixed)
        u_ref, (eps_ref, sig_ref), ny_ref = ref_path[k]
        assert rel_l2(host(u), u_ref) <= 1e-8
        h = host(hist).reshape(12, 8, om.n_cells)
        szz = h[6 + 2].mean()
        closed = float(np.clip(sig_prev + E_ * (strains[k] - e_prev), -sy, sy))
        assert abs(szz - closed) <= 1e-8 * sy, (k, szz, closed)
        assert np.abs(h[6 + 2] - closed).max() <= 1e-8 * sy
        trial = sig_prev + E_ * (strains[k] - e_prev)
        if abs(abs(trial) - sy) > 1e-9 * sy:  # at the exact yield point rounding decides
            assert st["n_yield"] == ny_ref
        sig_prev, e_prev = closed, strains[k]


def test_not_converged_keeps_the_history():
    n = 2
    mask, ubars, _, _ = inputs.j2_uniaxial(n=n)
    F = fem()
    m = F.fem_mesh(n, n, n)
    mat = F.j2_material(E, NU, SY)
    u = torch.zeros(3 * (n + 1) ** 3, dtype=torch.float64, device="cuda")
    hist = F.j2_history(m)
    with pytest.raises(F.FemError) as e:
        F.fem_j2_step(m, mat, dev(mask), dev(ubars[5]), u, hist, newton_maxit=0)
    assert e.value.status == F.FEM_ERR_NOT_CONVERGED
    assert float(hist.abs().max()) == 0.0


def test_non_finite_prescribed_value_is_reported():
    n = 2
    mask, ubars, _, _ = inputs.j2_uniaxial(n=n)
    F = fem()
    m = F.fem_mesh(n, n, n)
    ub = np.array(ubars[0])
    ub[np.flatnonzero(mask)[-1]] = np.nan
    u = torch.zeros(3 * (n + 1) ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FemError) as e:
        F.fem_j2_step(m, F.j2_material(E, NU, SY), dev(mask), dev(ub), u, F.j2_history(m))
    assert e.value.status == F.FEM_ERR_NONFINITE
