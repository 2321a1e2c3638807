"""Failure detection without a GPU fault: every condition ends in a status
code read on the host, and the CUDA context stays usable afterwards."""
import pytest
import torch

from paper_2212_00964_gb300 import inputs
from tests.gpu_common import dev, fem

pytestmark = pytest.mark.gpu


def still_usable(F):
    m = F.fem_mesh(2, 2, 2)
    u = torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda")
    y = F.fem_tangent_apply(m, F.material(0, 1.0, 0.3), u, torch.ones_like(u))
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()


def solve(F, w, **opt):
    m = F.fem_mesh(w.nx, w.ny, w.nz)
    u = torch.zeros(w.n_dofs, dtype=torch.float64, device="cuda")
    st = F.fem_solve(m, F.material(w.kind, w.E, w.nu), dev(w.mask), dev(w.u_bar), u, n_steps=w.n_steps,
                     options=F.default_options(**opt), check=False)
    return st


def test_inverted_element_reported():
    F = fem()
    w = inputs.c1(n=2, n_steps=1)
    w.mask, w.u_bar = inputs.clamp_and_compress(2, 2, 2, -0.95)
    st = solve(F, w)
    assert st["rc"] in (F.FEM_ERR_INVERTED, F.FEM_ERR_BREAKDOWN, F.FEM_ERR_NONFINITE)
    still_usable(F)


def test_newton_iteration_limit():
    F = fem()
    w = inputs.c1(n=3, n_steps=1)
    st = solve(F, w, newton_maxit=1, newton_rtol=1e-14)
    assert st["rc"] == F.FEM_ERR_NOT_CONVERGED
    still_usable(F)


def test_watchdog_timeout():
    F = fem()
    w = inputs.c1(n=8, n_steps=10)
    st = solve(F, w, timeout_s=1e-9)
    assert st["rc"] == F.FEM_ERR_TIMEOUT
    still_usable(F)


def test_invalid_arguments_rejected():
    F = fem()
    m = F.fem_mesh(2, 2, 2)
    u = torch.zeros(m.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FemError) as e:
        F.fem_tangent_apply(m, F.material(0, -1.0, 0.3), u, u.clone())
    assert e.value.status == F.FEM_ERR_ARG
    with pytest.raises(F.FemError):
        F.fem_solve(m, F.material(2, 1.0, 0.3), torch.zeros(m.n_dofs, dtype=torch.uint8, device="cuda"),
                    torch.zeros_like(u), u, n_steps=0)
    still_usable(F)
