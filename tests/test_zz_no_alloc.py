"""fem_solve_static, the allocation-free solve (no paper counterpart).

Some callers cannot allocate device memory when they solve: a process whose
GPU memory belongs to another framework's caching allocator, a real-time loop
that forbids allocation after start-up, or code running beside a global-mode
stream capture, which makes cudaMalloc illegal in every thread of the
process.  fem_solve_static serves them from a fixed static device array.

These tests call it through the C-ABI and check
  * its solutions against the FP64 oracle, twice in a row and interleaved
    with another problem (the array keeps the previous call's contents);
  * against fem_solve on the same inputs;
  * that a call after the first leaves the device's free memory unchanged;
  * that it runs, and solves correctly, on a side stream while another
    thread holds a global-mode stream capture open, and that the capture
    stays valid;
  * that a box beyond the array is refused with FEM_ERR_ARG.
The file is named so that pytest collects it last; it also passes alone in a
fresh process.
"""
import threading

import pytest
import torch

import oracle
from oracle import solve as osolve
from paper_2212_00964_gb300 import inputs
from tests.gpu_common import TOL_REFINED, dev, fem, host, rel_l2

pytestmark = pytest.mark.gpu


def oracle_solution(w):
    om = oracle.mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    omat = oracle.Material(w.kind, w.E, w.nu, w.simp_p, w.simp_emin)
    if w.kind == oracle.NEOHOOKE:
        return osolve.newton_solve(om, omat, w.mask, w.u_bar, w.point_load, w.cell_param, n_steps=w.n_steps)
    return osolve.linear_solve(om, omat, w.mask, w.u_bar, w.point_load, w.cell_param)


class StaticCase:
    """Device inputs of one workload, allocated once so that the calls under
    test allocate nothing themselves."""

    def __init__(self, F, w):
        self.w = w
        self.mat = F.material(w.kind, w.E, w.nu, w.simp_p, w.simp_emin)
        self.mask, self.ubar = dev(w.mask), dev(w.u_bar)
        self.f = dev(w.point_load) if w.point_load is not None else None
        self.cp = dev(w.cell_param) if w.cell_param is not None else None
        self.u = torch.zeros(w.n_dofs, dtype=torch.float64, device="cuda")

    def solve(self, F, opt, stream=None):
        w = self.w
        self.u.zero_()
        return F.fem_solve_static(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz, self.mat, self.mask, self.ubar, self.u,
                                  self.f, self.cp, w.n_steps, opt, stream=stream, check=False)


def test_static_solve_matches_oracle_on_consecutive_calls():
    F = fem()
    opt = F.default_options(newton_rtol=1e-12)
    nh = StaticCase(F, inputs.c1(n=12, n_steps=3))
    simp = StaticCase(F, inputs.c2(nx=12, ny=6, nz=6))
    ref_nh, ref_simp = oracle_solution(nh.w), oracle_solution(simp.w)
    for _ in range(2):
        assert nh.solve(F, opt)["status"] == 0
        assert rel_l2(host(nh.u), ref_nh) <= TOL_REFINED
    assert simp.solve(F, opt)["status"] == 0
    assert rel_l2(host(simp.u), ref_simp) <= TOL_REFINED
    assert nh.solve(F, opt)["status"] == 0
    assert rel_l2(host(nh.u), ref_nh) <= TOL_REFINED


def test_static_solve_matches_fem_solve():
    F = fem()
    opt = F.default_options(newton_rtol=1e-12)
    c = StaticCase(F, inputs.c1(n=12, n_steps=3))
    m = F.fem_mesh(c.w.nx, c.w.ny, c.w.nz)
    u = torch.zeros_like(c.u)
    F.fem_solve(m, c.mat, c.mask, c.ubar, u, None, None, c.w.n_steps, opt)
    assert c.solve(F, opt)["status"] == 0
    assert rel_l2(host(c.u), host(u)) <= TOL_REFINED


def test_static_solve_fp64_matches_oracle():
    F = fem()
    opt = F.default_options(precision=F.FEM_FP64, newton_rtol=1e-12, pcg_rtol=1e-8)
    c = StaticCase(F, inputs.c1(n=6, n_steps=2))
    ref = oracle_solution(c.w)
    for _ in range(2):
        assert c.solve(F, opt)["status"] == 0
        assert rel_l2(host(c.u), ref) <= TOL_REFINED


def test_static_solve_leaves_free_device_memory_unchanged():
    F = fem()
    opt = F.default_options(newton_rtol=1e-12)
    c = StaticCase(F, inputs.c1(n=10, n_steps=2))
    assert c.solve(F, opt)["status"] == 0  # first call: module loading, symbol lookup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert c.solve(F, opt)["status"] == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes across two calls"


def test_static_solve_beside_a_global_mode_capture():
    """A second thread begins a global-mode stream capture (as
    torch.cuda.graph does by default) and holds it open while this thread
    solves on its own stream; the solve must succeed and be correct, and the
    other thread's capture must still end in a valid graph."""
    F = fem()
    opt = F.default_options(newton_rtol=1e-12)
    c = StaticCase(F, inputs.c1(n=8, n_steps=2))
    ref = oracle_solution(c.w)
    assert c.solve(F, opt)["status"] == 0  # set-up call before any capture
    side = torch.cuda.Stream()
    cap_stream = torch.cuda.Stream()
    x = torch.zeros(64, device="cuda")
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    opened, solved = threading.Event(), threading.Event()
    err = []

    def capturer():
        try:
            with torch.cuda.stream(cap_stream):
                graph.capture_begin(capture_error_mode="global")
                x.add_(1.0)
                opened.set()
                solved.wait(timeout=120)
                graph.capture_end()
        except Exception as e:  # reported by the main thread
            err.append(e)
            opened.set()

    c.u.zero_()
    torch.cuda.synchronize()
    t = threading.Thread(target=capturer)
    t.start()
    assert opened.wait(timeout=60)
    w = c.w
    st = F.fem_solve_static(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz, c.mat, c.mask, c.ubar, c.u, c.f, c.cp,
                            w.n_steps, opt, stream=side, check=False)
    solved.set()
    t.join(timeout=120)
    assert not err, f"the capture in the other thread failed: {err[0]}"
    assert st["rc"] == 0 and st["status"] == 0, st
    graph.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
    assert rel_l2(host(c.u), ref) <= TOL_REFINED


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
