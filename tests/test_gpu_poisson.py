"""GPU parity of the scalar Poisson path (full-field inference, Sec. 3.1):
the stiffness and mass stencils (fem_poisson_apply), Jacobi-PCG
(fem_poisson_solve) and the objective with its adjoint gradient
(fem_poisson_gradient) against the oracle, on ragged boxes and at the
paper's 50x50x10 size, plus the Taylor test of Eqs. (27)-(28) and the
inference loop through the GPU gradient."""
import numpy as np
import pytest
import torch

import oracle
from oracle import poisson as op
from paper_2212_00964_gb300 import inputs
from tests.gpu_common import dev, fem, host, rel_l2

pytestmark = pytest.mark.gpu

BOXES = [(3, 4, 2, 1.0, 1.3, 0.4), (1, 2, 1, 0.5, 1.0, 0.2), (37, 5, 3, 2.0, 0.3, 0.9)]


@pytest.mark.parametrize("box", BOXES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_and_mass_parity(box, prec):
    nx, ny, nz, lx, ly, lz = box
    F = fem()
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 1e-5
    m = F.fem_mesh(nx, ny, nz, lx, ly, lz)
    om = oracle.mesh(nx, ny, nz, lx, ly, lz)
    rng = np.random.default_rng(nx + ny + nz)
    x = rng.standard_normal(om.n_nodes)
    mask = (rng.uniform(size=om.n_nodes) < 0.3).astype(np.uint8)
    alpha = 1.3
    A, M = op.assemble(om, alpha)
    y = F.fem_poisson_apply(m, dev(x, dt), alpha)
    assert rel_l2(host(y), A @ x) <= tol
    y = F.fem_poisson_apply(m, dev(x, dt), alpha, F.FEM_POISSON_MASS)
    assert rel_l2(host(y), M @ x) <= tol
    y = F.fem_poisson_apply(m, dev(x, dt), alpha, F.FEM_POISSON_STIFFNESS, dev(mask))
    assert rel_l2(host(y), op.apply(om, alpha, x, mask)) <= tol
    y = F.fem_poisson_apply(m, dev(x, dt), alpha, F.FEM_POISSON_MASS, dev(mask))
    assert rel_l2(host(y), op.load(om, x, mask)) <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_solve_paper_size(prec):
    """A u = M theta_true on the 50x50x10 box: CG against the oracle's LU."""
    w = inputs.poisson_inference()
    F = fem()
    dt = torch.float64 if prec == "fp64" else torch.float32
    m = F.fem_mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    om, prob = op.from_workload(w)
    ref = prob.solve(w.theta_true)
    b = F.fem_poisson_apply(m, dev(w.theta_true, dt), w.alpha, F.FEM_POISSON_MASS, dev(w.mask))
    rtol = 1e-12 if prec == "fp64" else 1e-6
    u, it, res = F.fem_poisson_solve(m, b, w.alpha, dev(w.mask), rtol=rtol, maxit=5000)
    assert 0 < it < 5000 and res <= rtol
    assert rel_l2(host(u), ref) <= (1e-9 if prec == "fp64" else 1e-4)
    assert np.all(host(u)[w.mask == 1] == 0)


def test_mixed_precision_solve_and_gradient():
    """FP32 CG under FP64 refinement reaches the FP64 answer at the paper's size."""
    w = inputs.poisson_inference()
    F = fem()
    m = F.fem_mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    om, prob = op.from_workload(w)
    b = F.fem_poisson_apply(m, dev(w.theta_true), w.alpha, F.FEM_POISSON_MASS, dev(w.mask))
    u, it, res = F.fem_poisson_solve(m, b, w.alpha, dev(w.mask), rtol=1e-11, maxit=20000, mixed=True)
    assert res <= 1e-11 and it > 0
    assert rel_l2(host(u), prob.solve(w.theta_true)) <= 1e-8
    rng = np.random.default_rng(8)
    theta = rng.standard_normal(om.n_nodes)
    u_obs = 0.01 * rng.standard_normal(w.obs.size)
    J, g, _, _ = prob.gradient(theta, w.obs, u_obs)
    out = F.fem_poisson_gradient(m, dev(theta), dev(w.obs), dev(u_obs), w.alpha, dev(w.mask), rtol=1e-11,
                                 maxit=20000, mixed=True)
    assert abs(out["J"] - J) <= 1e-8 * abs(J)
    assert rel_l2(host(out["grad"]), g) <= 1e-7


def test_gradient_parity_small_and_paper_size():
    for w in (inputs.poisson_inference(4, 4, 3, 1.0, 1.0, 0.2, n_obs=6, seed=3), inputs.poisson_inference()):
        F = fem()
        m = F.fem_mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
        om, prob = op.from_workload(w)
        rng = np.random.default_rng(7)
        theta = rng.standard_normal(om.n_nodes)
        u_obs = prob.solve(w.theta_true)[w.obs] + 0.01 * rng.standard_normal(w.obs.size)
        J, g, u, lam = prob.gradient(theta, w.obs, u_obs)
        out = F.fem_poisson_gradient(m, dev(theta), dev(w.obs), dev(u_obs), w.alpha, dev(w.mask), rtol=1e-13,
                                     maxit=20000)
        assert abs(out["J"] - J) <= 1e-9 * abs(J)
        assert rel_l2(host(out["u"]), u) <= 1e-9
        assert rel_l2(host(out["lam"]), lam) <= 1e-8
        assert rel_l2(host(out["grad"]), g) <= 1e-8
        assert out["iters"][0] > 0 and out["iters"][1] > 0


def test_gradient_taylor_rates():
    """Eqs. (27)-(28) with the GPU objective and gradient (FP64)."""
    w = inputs.poisson_inference(10, 10, 4, 1.0, 1.0, 0.2, n_obs=20, seed=5)
    F = fem()
    m = F.fem_mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    rng = np.random.default_rng(9)
    theta = rng.standard_normal(m.n_nodes)
    dth = rng.standard_normal(m.n_nodes)
    u_obs = 0.01 * rng.standard_normal(w.obs.size)

    def run(t):
        return F.fem_poisson_gradient(m, dev(t), dev(w.obs), dev(u_obs), w.alpha, dev(w.mask), rtol=1e-14,
                                      maxit=20000)

    base = run(theta)
    slope = float(host(base["grad"]) @ dth)
    hs = np.array([1e-3, 1e-2, 1e-1])
    r0, r1 = [], []
    for h in hs:
        Jh = run(theta + h * dth)["J"]
        r0.append(abs(Jh - base["J"]))
        r1.append(abs(Jh - base["J"] - h * slope))
    s0 = np.diff(np.log10(r0)) / np.diff(np.log10(hs))
    s1 = np.diff(np.log10(r1)) / np.diff(np.log10(hs))
    assert np.all(np.abs(s0 - 1) < 0.1) and np.all(np.abs(s1 - 2) < 0.1), (s0, s1)


def test_inference_loop_with_gpu_gradient():
    """20 L-BFGS iterations (scipy, host) on the GPU objective and gradient at
    the paper's size: the same drop of the objective and the same error band
    as the oracle's loop."""
    from scipy.optimize import minimize
    w = inputs.poisson_inference()
    F = fem()
    m = F.fem_mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    om, prob = op.from_workload(w)
    U = prob.solve(w.theta_true)
    obs_d, uobs_d, mask_d = dev(w.obs), dev(U[w.obs]), dev(w.mask)
    hist = []

    def fun(t):
        out = F.fem_poisson_gradient(m, dev(t), obs_d, uobs_d, w.alpha, mask_d, rtol=1e-12, maxit=20000)
        hist.append(out["J"])
        return out["J"], host(out["grad"])

    res = minimize(fun, np.zeros(om.n_nodes), jac=True, method="L-BFGS-B",
                   options={"maxiter": 20, "gtol": 0.0, "ftol": 0.0})
    err = prob.rel_l2_error(prob.solve(res.x), U)
    assert min(hist) < 1e-4 * hist[0]
    assert 0.06 <= err <= 0.24


@pytest.mark.parametrize("mixed", [False, True])
def test_autograd_solve_matches_the_adjoint_gradient(mixed):
    """torch autograd through PoissonSolve (forward: mass + CG; backward:
    fem_poisson_adjoint) gives the oracle's gradient of the objective of
    Eq. (26) written as plain torch ops on u."""
    from paper_2212_00964_gb300.autograd import PoissonSolve
    w = inputs.poisson_inference(12, 10, 4, 1.0, 1.0, 0.2, n_obs=30, seed=6)
    F = fem()
    m = F.fem_mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    om, prob = op.from_workload(w)
    rng = np.random.default_rng(10)
    theta = rng.standard_normal(om.n_nodes)
    u_obs = 0.01 * rng.standard_normal(w.obs.size)
    J_ref, g_ref, _, _ = prob.gradient(theta, w.obs, u_obs)
    solve = PoissonSolve(m, w.alpha, dev(w.mask), rtol=1e-12, mixed=mixed)
    th = dev(theta).requires_grad_(True)
    u = solve(th)
    J = ((u[dev(w.obs)] - dev(u_obs)) ** 2).sum()
    J.backward()
    assert abs(float(J.detach()) - J_ref) <= 1e-9 * J_ref
    assert rel_l2(host(th.grad), g_ref) <= 1e-8


def test_bad_observation_index_is_an_argument_error():
    w = inputs.poisson_inference(4, 4, 3, 1.0, 1.0, 0.2, n_obs=6, seed=3)
    F = fem()
    m = F.fem_mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    obs = w.obs.copy()
    obs[2] = m.n_nodes + 5
    with pytest.raises(F.FemError) as e:
        F.fem_poisson_gradient(m, dev(np.ones(m.n_nodes)), dev(obs), dev(np.zeros(obs.size)), 1.0, dev(w.mask))
    assert e.value.status == F.FEM_ERR_ARG
    # the handle stays usable
    y = F.fem_poisson_apply(m, dev(np.ones(m.n_nodes)), 1.0)
    assert abs(float(y.sum())) <= 1e-12


def test_non_finite_right_hand_side_is_reported():
    w = inputs.poisson_inference(6, 5, 3, 1.0, 1.0, 0.2, n_obs=5, seed=2)
    F = fem()
    m = F.fem_mesh(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz)
    b = np.zeros(m.n_nodes)
    b[int(np.flatnonzero(w.mask == 0)[0])] = np.nan
    for mixed in (False, True):
        with pytest.raises(F.FemError) as e:
            F.fem_poisson_solve(m, dev(b), w.alpha, dev(w.mask), mixed=mixed)
        assert e.value.status == F.FEM_ERR_NONFINITE
