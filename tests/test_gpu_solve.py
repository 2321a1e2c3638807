"""GPU parity of the solvers against the oracle's Newton / spsolve solutions:
the linear-elastic c0 solve (FP64 and mixed), Neo-Hookean load-stepped
Newton (FP64 and mixed with FP64 refinement) up to 17^3, SIMP solve, and
the 64^3 Neo-Hookean benchmark solve checked by properties that hold at any
size (mixed vs FP64 GPU solution, oracle FP64 residual at the GPU
solution)."""
import functools

import numpy as np
import pytest
import torch

import oracle
from oracle import solve as osolve
from paper_2212_00964_gb300 import inputs
from tests.gpu_common import TOL_FP64, TOL_REFINED, dev, fem, host, rel_l2

pytestmark = pytest.mark.gpu


def gpu_solve(w, precision, f_ext=None, **opt):
    F = fem()
    m = F.fem_mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    if f_ext is None and w.traction is not None:
        f = torch.zeros(w.n_dofs, dtype=torch.float64, device="cuda")
        F.fem_load_traction(m, w.traction[0], w.traction[1], f)
    elif f_ext is not None:
        f = dev(f_ext)
    elif w.point_load is not None:
        f = dev(w.point_load)
    else:
        f = None
    u = torch.zeros(w.n_dofs, dtype=torch.float64, device="cuda")
    o = F.default_options(precision=precision, **opt)
    cp = None if w.cell_param is None else dev(w.cell_param)
    st = F.fem_solve(m, F.material(w.kind, w.E, w.nu, w.simp_p, w.simp_emin), dev(w.mask), dev(w.u_bar), u,
                     f, cp, w.n_steps, o)
    return host(u), st


def oracle_solve(w):
    om = oracle.mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    mat = oracle.Material(w.kind, w.E, w.nu, w.simp_p, w.simp_emin)
    f = None
    if w.traction is not None:
        f = oracle.traction(om, *w.traction)
    elif w.point_load is not None:
        f = w.point_load
    if w.kind == oracle.NEOHOOKE:
        return osolve.newton_solve(om, mat, w.mask, w.u_bar, f, w.cell_param, n_steps=w.n_steps)
    return osolve.linear_solve(om, mat, w.mask, w.u_bar, f, w.cell_param)


@functools.lru_cache(None)
def oracle_c1(n):
    return oracle_solve(inputs.c1(n=n, n_steps=10))


def test_c0_linear_elastic_fp64():
    w = inputs.c0()
    ref = oracle_solve(w)
    u, st = gpu_solve(w, 0, newton_rtol=1e-13, pcg_rtol=1e-10)
    assert st["status"] == 0
    assert rel_l2(u, ref) <= TOL_FP64


def test_c0_linear_elastic_mixed_refined():
    w = inputs.c0()
    ref = oracle_solve(w)
    u, st = gpu_solve(w, 2, newton_rtol=1e-12)
    assert st["status"] == 0 and st["newton_iters"] >= 2  # FP32 CG + FP64 refinement sweeps
    assert rel_l2(u, ref) <= TOL_REFINED


@pytest.mark.parametrize("apply_kernel", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12])
@pytest.mark.parametrize("n", [4, 8, 9])
def test_neohooke_load_steps(n, apply_kernel):
    """Every CG apply kernel (per-cell scatter at 3 and 4 CTAs/SM, 8x4x4
    bricks, per-cell on stored tangent data, packed Gauss-point pairs with
    and without stored data; FP64 runs the scalar kernel of the same data);
    9^3 leaves ragged bricks in every direction and a ragged last cell tile."""
    w = inputs.c1(n=n, n_steps=10)
    ref = oracle_c1(n)
    u64, st64 = gpu_solve(w, 0, newton_rtol=1e-13, pcg_rtol=1e-8, apply_kernel=apply_kernel)
    assert st64["status"] == 0 and st64["load_steps"] == 10 and st64["apply_kernel"] == apply_kernel
    assert rel_l2(u64, ref) <= TOL_FP64
    u32, st32 = gpu_solve(w, 2, newton_rtol=1e-12, apply_kernel=apply_kernel)
    assert st32["status"] == 0 and st32["apply_kernel"] == apply_kernel
    assert rel_l2(u32, ref) <= TOL_REFINED


@pytest.mark.slow
def test_c1_17cube_against_the_oracle():
    """17^3 Neo-Hookean, 10 load steps (17,496 DOF; 4,913 cells, 38 full
    cell tiles and a ragged one; many CG chunks per Newton iteration): the
    default solves (autotuned apply kernel, adaptive inner tolerance, one
    graph launch with device-side loops) equal the oracle's Newton / spsolve
    solution, mixed to 1e-8 and all-FP64 to 1e-10 (about two minutes of
    oracle time on one core)."""
    n = 17
    w = inputs.c1(n=n, n_steps=10)
    ref = oracle_c1(n)
    u32, st32 = gpu_solve(w, 2, newton_rtol=1e-12)
    assert st32["status"] == 0 and st32["load_steps"] == 10
    assert rel_l2(u32, ref) <= TOL_REFINED
    u64, st64 = gpu_solve(w, 0, newton_rtol=1e-13, pcg_rtol=1e-8)
    assert st64["status"] == 0 and st64["load_steps"] == 10
    assert rel_l2(u64, ref) <= TOL_FP64


@pytest.mark.parametrize("apply_kernel", [8, 9])
@pytest.mark.parametrize("n", [8, 9])
def test_packed_kernels_at_64_cells_per_block(n, apply_kernel):
    """fem_options.cta_cells = 64: the packed CG kernels iterate over half
    tiles of the stored-data layout (9^3: ragged last half tile); same bar
    as at 128 cells per block, and the stats report the block size."""
    w = inputs.c1(n=n, n_steps=10)
    ref = oracle_c1(n)
    u32, st32 = gpu_solve(w, 2, newton_rtol=1e-12, apply_kernel=apply_kernel, cta_cells=64)
    assert st32["status"] == 0 and st32["apply_kernel"] == apply_kernel and st32["cta_cells"] == 64
    assert rel_l2(u32, ref) <= TOL_REFINED


def test_cells_per_block_option_is_checked():
    F = fem()
    with pytest.raises(F.FemError) as ei:
        gpu_solve(inputs.c1(n=4, n_steps=1), 2, cta_cells=96)
    assert ei.value.status == -1  # FEM_ERR_ARG


def test_neohooke_noncubic_with_stiffness_field():
    w = inputs.c1(n=4, n_steps=3)
    w.nx, w.ny, w.nz = 6, 4, 3
    w.lx, w.ly, w.lz = 1.5, 1.0, 0.75
    w.mask, w.u_bar = inputs.clamp_and_compress(6, 4, 3, -0.1)
    w.cell_param = np.random.default_rng(4).lognormal(0, 0.5, 6 * 4 * 3)
    ref = oracle_solve(w)
    u, st = gpu_solve(w, 2, newton_rtol=1e-12)
    assert st["status"] == 0
    assert rel_l2(u, ref) <= TOL_REFINED


@pytest.mark.parametrize("apply_kernel", [1, 2, 3, 8, 11])
def test_simp_cantilever_small(apply_kernel):
    w = inputs.c2(nx=16, ny=8, nz=8)
    ref = oracle_solve(w)
    u, st = gpu_solve(w, 2, newton_rtol=1e-12, apply_kernel=apply_kernel)
    assert st["status"] == 0
    assert rel_l2(u, ref) <= TOL_REFINED
    u64, st64 = gpu_solve(w, 0, newton_rtol=1e-13, pcg_rtol=1e-9, apply_kernel=apply_kernel)
    assert rel_l2(u64, ref) <= TOL_FP64


def test_simp_full_size_tensor_core_apply():
    """The 128x64x64 SIMP cantilever (4,096 cell tiles, several per CTA) with
    the CG apply on the tensor cores (kernel 11, split-TF32 shared element
    matrix) and on the CUDA cores (kernel 8): the same FP64-refined solution,
    and about as many refinement sweeps and CG iterations as the FP32 apply
    needs (an apply less accurate than FP32 would slow both)."""
    w = inputs.c2()
    u8, st8 = gpu_solve(w, 2, newton_rtol=1e-10, apply_kernel=8)
    u11, st11 = gpu_solve(w, 2, newton_rtol=1e-10, apply_kernel=11)
    assert st8["status"] == 0 and st11["status"] == 0 and st11["apply_kernel"] == 11
    assert rel_l2(u11, u8) <= 1e-8
    assert st11["newton_iters"] <= st8["newton_iters"] + 1
    # CG counts of one configuration vary by about +-7 % between runs (atomic
    # summation order, adaptive inner tolerance); a less accurate apply cost
    # 20-40 % more
    assert st11["pcg_iters"] <= 1.25 * st8["pcg_iters"]


def test_tensor_core_kernel_needs_one_linear_instance():
    """Apply kernel 11 is refused for a Neo-Hookean problem (argument error)."""
    F = fem()
    with pytest.raises(F.FemError) as ei:
        gpu_solve(inputs.c1(n=4, n_steps=1), 2, apply_kernel=11)
    assert ei.value.status == -1  # FEM_ERR_ARG


@pytest.mark.parametrize("n", [8, 9])
@pytest.mark.parametrize("apply_kernel", [1, 5])
def test_fused_cg_kernel(apply_kernel, n):
    """cg_fused = 1: one kernel per CG iteration (the update of iteration
    k-1 recomputed per node inside the apply of iteration k, owners writing
    the vectors); same parity bar as the two-kernel CG."""
    w = inputs.c1(n=n, n_steps=10)
    ref = oracle_c1(n)
    u32, st32 = gpu_solve(w, 2, newton_rtol=1e-12, apply_kernel=apply_kernel, cg_fused=1)
    assert st32["status"] == 0 and st32["apply_kernel"] == apply_kernel
    assert rel_l2(u32, ref) <= TOL_REFINED


def test_stored_tangent_kernel_needs_neohooke():
    """Apply kernel 4 is refused (argument error, nothing launched) for a
    linear-elastic problem."""
    w = inputs.c0()
    F = fem()
    with pytest.raises(F.FemError) as ei:
        gpu_solve(w, 2, apply_kernel=4)
    assert ei.value.status == -1  # FEM_ERR_ARG


def test_deterministic_repeat():
    """Same inputs, same launch configuration: solution equal to round-off
    of the atomics order (and the FP64 residual drives both to 1e-12)."""
    w = inputs.c1(n=6, n_steps=2)
    a, _ = gpu_solve(w, 2, newton_rtol=1e-12)
    b, _ = gpu_solve(w, 2, newton_rtol=1e-12)
    assert rel_l2(a, b) <= 1e-9


@pytest.mark.slow
def test_c1_full_size_mixed_vs_fp64_and_oracle_residual():
    """64^3 Neo-Hookean, 10 load steps: the mixed solution equals the all-FP64
    GPU solution to 1e-8, and the oracle's FP64 residual at the mixed
    solution is at the Newton tolerance (a property that holds at any size)."""
    w = inputs.c1()
    u32, st32 = gpu_solve(w, 2, newton_rtol=1e-10)
    assert st32["status"] == 0 and st32["load_steps"] == 10
    u64, st64 = gpu_solve(w, 0, newton_rtol=1e-10, pcg_rtol=1e-6)
    assert st64["status"] == 0
    assert rel_l2(u32, u64) <= TOL_REFINED
    om = oracle.mesh(w.nx, w.ny, w.nz)
    R = oracle.residual(om, oracle.Material(w.kind, w.E, w.nu), u32, None, None, w.mask)
    assert np.linalg.norm(R) <= 1e-9 * st32["ref_rnorm"]


@pytest.mark.parametrize("graph_loop", [0, 1])
def test_graph_loop_modes_agree(graph_loop):
    """The one-graph solve (device-side loops over Newton rounds and CG
    chunks) and the host-driven loop reach the oracle's solution, with the
    same iteration counts up to CG rounding."""
    n = 8
    w = inputs.c1(n=n, n_steps=10)
    ref = oracle_c1(n)
    u, st = gpu_solve(w, 2, newton_rtol=1e-12, graph_loop=graph_loop)
    assert st["status"] == 0 and st["load_steps"] == 10
    assert rel_l2(u, ref) <= TOL_REFINED
