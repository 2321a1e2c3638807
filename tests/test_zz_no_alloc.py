"""fem_solve_static, the allocation-free solve (no paper counterpart).

Some callers cannot allocate device memory when they solve: a process whose
GPU memory belongs to another framework's caching allocator, a real-time loop
that forbids allocation after start-up, or code running inside a global-mode
stream capture.  fem_solve_static serves them from a fixed static device
array.  These tests call it through the C-ABI and compare it with fem_solve on
the same inputs, twice in a row and interleaved with another problem (the
array keeps the previous call's contents).  The file is named so that pytest
collects it last; it also passes alone in a fresh process.
"""
import pytest
import torch

from paper_2212_00964_gb300 import inputs
from tests.gpu_common import TOL_REFINED, dev, fem, host, rel_l2

pytestmark = pytest.mark.gpu


def reference_solve(F, w, opt):
    m = F.fem_mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    u = torch.zeros(w.n_dofs, dtype=torch.float64, device="cuda")
    f = dev(w.point_load) if w.point_load is not None else None
    cp = dev(w.cell_param) if w.cell_param is not None else None
    F.fem_solve(m, F.material(w.kind, w.E, w.nu, w.simp_p, w.simp_emin), dev(w.mask), dev(w.u_bar), u, f, cp,
                w.n_steps, opt)
    return host(u)


def static_solve(F, w, opt):
    u = torch.zeros(w.n_dofs, dtype=torch.float64, device="cuda")
    f = dev(w.point_load) if w.point_load is not None else None
    cp = dev(w.cell_param) if w.cell_param is not None else None
    st = F.fem_solve_static(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz,
                            F.material(w.kind, w.E, w.nu, w.simp_p, w.simp_emin), dev(w.mask), dev(w.u_bar), u,
                            f, cp, w.n_steps, opt)
    assert st["status"] == 0
    return host(u)


def test_static_solve_matches_fem_solve_on_consecutive_calls():
    F = fem()
    opt = F.default_options(newton_rtol=1e-12)
    nh = inputs.c1(n=12, n_steps=3)
    simp = inputs.c2(nx=12, ny=6, nz=6)
    ref_nh = reference_solve(F, nh, opt)
    ref_simp = reference_solve(F, simp, opt)
    for _ in range(2):
        assert rel_l2(static_solve(F, nh, opt), ref_nh) <= TOL_REFINED
    assert rel_l2(static_solve(F, simp, opt), ref_simp) <= TOL_REFINED
    assert rel_l2(static_solve(F, nh, opt), ref_nh) <= TOL_REFINED


def test_static_solve_fp64_matches():
    F = fem()
    opt = F.default_options(precision=F.FEM_FP64, newton_rtol=1e-12, pcg_rtol=1e-8)
    w = inputs.c1(n=6, n_steps=2)
    ref = reference_solve(F, w, opt)
    for _ in range(2):
        assert rel_l2(static_solve(F, w, opt), ref) <= TOL_REFINED


def test_static_solve_rejects_meshes_beyond_the_array():
    F = fem()
    n = 64
    D = 3 * (n + 1) ** 3
    u = torch.zeros(D, dtype=torch.float64, device="cuda")
    mask = torch.zeros(D, dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FemError) as e:
        F.fem_solve_static(n, n, n, 1.0, 1.0, 1.0, F.material(2, 10.0, 0.3), mask, torch.zeros_like(u), u,
                           n_steps=1)
    assert e.value.status == F.FEM_ERR_ARG
    assert "static array" in str(e.value)
