"""Batched launcher: many Neo-Hookean instances of uneven size and material
in one graph-captured launch sequence; each instance against the oracle and
against its own single-instance GPU solve."""
import numpy as np
import pytest
import torch

import oracle
from oracle import solve as osolve
from paper_2212_00964_gb300 import inputs
from tests.gpu_common import TOL_REFINED, dev, fem, host, rel_l2

pytestmark = pytest.mark.gpu


def make_instances(F, works):
    meshes = {}
    insts = []
    for w in works:
        key = (w.nx, w.ny, w.nz)
        if key not in meshes:
            meshes[key] = F.fem_mesh(*key)
        insts.append(F.Instance(meshes[key], F.material(w.kind, w.E, w.nu), dev(w.mask), dev(w.u_bar),
                                torch.zeros(w.n_dofs, dtype=torch.float64, device="cuda"), w.n_steps))
    return insts


@pytest.mark.parametrize("apply_kernel", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12])
def test_small_batch_vs_oracle_and_single(apply_kernel):
    F = fem()
    works = inputs.c3(n_inst=7, seed=3, lo=2, hi=9, n_steps=3)
    insts = make_instances(F, works)
    rc, stats = F.fem_solve_batched(insts, F.default_options(newton_rtol=1e-12, apply_kernel=apply_kernel))
    assert rc == 0 and all(s["status"] == 0 for s in stats)
    for w, I, st in zip(works, insts, stats):
        om = oracle.mesh(w.nx, w.ny, w.nz)
        ref = osolve.newton_solve(om, oracle.Material(w.kind, w.E, w.nu), w.mask, w.u_bar, n_steps=w.n_steps)
        assert rel_l2(host(I.u), ref) <= TOL_REFINED
        assert st["load_steps"] == w.n_steps
        u1 = torch.zeros_like(I.u)
        F.fem_solve(I.mesh, I.mat, I.mask, I.u_bar, u1, n_steps=w.n_steps,
                    options=F.default_options(newton_rtol=1e-12))
        assert rel_l2(host(I.u), host(u1)) <= TOL_REFINED


@pytest.mark.parametrize("apply_kernel", [8, 9])
def test_small_batch_at_64_cells_per_block(apply_kernel):
    """Half-tile block iterations in a batch: the instance of each half tile
    is found from its 128-cell tile."""
    F = fem()
    works = inputs.c3(n_inst=7, seed=3, lo=2, hi=9, n_steps=3)
    insts = make_instances(F, works)
    rc, stats = F.fem_solve_batched(insts, F.default_options(newton_rtol=1e-12, apply_kernel=apply_kernel,
                                                             cta_cells=64))
    assert rc == 0 and all(s["status"] == 0 for s in stats)
    for w, I in zip(works, insts):
        om = oracle.mesh(w.nx, w.ny, w.nz)
        ref = osolve.newton_solve(om, oracle.Material(w.kind, w.E, w.nu), w.mask, w.u_bar, n_steps=w.n_steps)
        assert rel_l2(host(I.u), ref) <= TOL_REFINED


@pytest.mark.slow
def test_full_batch_256_instances():
    """The 256-instance workload (edges 8..32): every instance converges; the
    two smallest are checked against the oracle."""
    F = fem()
    works = inputs.c3()
    insts = make_instances(F, works)
    rc, stats = F.fem_solve_batched(insts, F.default_options(newton_rtol=1e-10))
    assert rc == 0, [s["status"] for s in stats if s["status"] != 0][:5]
    sizes = np.array([w.nx for w in works])
    for t in np.argsort(sizes, kind="stable")[:2]:
        w = works[t]
        om = oracle.mesh(w.nx, w.ny, w.nz)
        ref = osolve.newton_solve(om, oracle.Material(w.kind, w.E, w.nu), w.mask, w.u_bar, n_steps=w.n_steps,
                                  rtol=1e-10)
        assert rel_l2(host(insts[t].u), ref) <= TOL_REFINED
