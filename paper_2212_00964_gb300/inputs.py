"""Seeded synthetic workloads for the HEX8 weak-form path.

This module holds no arithmetic of the finite-element method: it only
describes problems (box sizes, material constants, which DOFs are
prescribed and to what, load specifications, seeded random fields).  Both the
CUDA path and the CPU oracle consume what it returns, each computing loads and
operators on its own.

Workloads (structured unit-cube boxes standing in for the paper's missing
cylinder / dog-bone meshes, at the paper's 3D solid-mechanics DOF scale):
  c0  linear elasticity 8^3, E=70e3, nu=0.3, x=0 clamped, traction (0,0,-100)
      on x=1, one linear solve;
  c1  Neo-Hookean 64^3, E=10, nu=0.3, x=0 clamped, u_x=-0.1 on x=1,
      10 load steps;
  c2  SIMP cantilever 128x64x64 on a 2x1x1 box, theta ~ U[0.01,1] (seed 2),
      E(theta) = 1e-3 + theta^3 (1 - 1e-3), nu=0.3, x=0 clamped, total force
      (0,0,-1) spread over a 4x4 node patch at the bottom of the x=2 face;
  c3  256 Neo-Hookean instances, edge n ~ U{8..32}, E log-uniform [1e2,1e4],
      nu ~ U[0.2,0.45], compression ~ U[0.02,0.15], 10 load steps (seed 3);
  c4  Neo-Hookean 128^3, stiffness scale log-normal(0, 0.5) (seed 4), E=10,
      nu=0.3, 5 load steps, face-displacement target ~ N(0, 0.02^2) (seed 5001).
Random streams are NumPy ``default_rng(seed)`` (PCG64), drawn once on the host.

Layout conventions (the C-ABI's): node id = i + (nx+1)(j + (ny+1)k), DOF
3*node + component, cell id = i + nx(j + ny k).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

LINEAR, SIMP, NEOHOOKE = 0, 1, 2


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    kind: int
    E: float
    nu: float
    simp_p: float = 3.0
    simp_emin: float = 1e-3
    n_steps: int = 1
    mask: Optional[np.ndarray] = None        # uint8 [D], 1 = prescribed
    u_bar: Optional[np.ndarray] = None       # float64 [D], final prescribed values
    point_load: Optional[np.ndarray] = None  # float64 [D], nodal forces (or None)
    traction: Optional[tuple] = None         # (face, (tx, ty, tz)) or None
    cell_param: Optional[np.ndarray] = None  # float64 [Ne] or None
    extra: dict = field(default_factory=dict)

    @property
    def n_nodes(self):
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_cells(self):
        return self.nx * self.ny * self.nz

    @property
    def n_dofs(self):
        return 3 * self.n_nodes


def node_index(nx, ny, nz, i, j, k):
    return i + (nx + 1) * (j + (ny + 1) * k)


def face_nodes(nx, ny, nz, face):
    """Node ids on a face of the box: 'x0','x1','y0','y1','z0','z1'."""
    I, J, K = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    sel = {"x0": I == 0, "x1": I == nx, "y0": J == 0, "y1": J == ny, "z0": K == 0, "z1": K == nz}[face]
    return np.sort(node_index(nx, ny, nz, I[sel], J[sel], K[sel]).astype(np.int64))


def dirichlet(nx, ny, nz, specs):
    """specs: list of (face, component, value).  Returns (mask u8[D], u_bar f64[D])."""
    D = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    mask = np.zeros(D, np.uint8)
    ubar = np.zeros(D, np.float64)
    for face, comp, val in specs:
        n = face_nodes(nx, ny, nz, face)
        mask[3 * n + comp] = 1
        ubar[3 * n + comp] = val
    return mask, ubar


def clamp_and_compress(nx, ny, nz, disp):
    """x=0 face fully clamped, u_x = disp on the x=1 face (u_y, u_z free there)."""
    return dirichlet(nx, ny, nz, [("x0", 0, 0.0), ("x0", 1, 0.0), ("x0", 2, 0.0), ("x1", 0, disp)])


def random_state(n_dofs, h, seed, scale=0.05):
    """Displacement u = scale * h * N(0,1) per DOF (det F > 0 for scale << 1)."""
    return scale * h * np.random.default_rng(seed).standard_normal(n_dofs)


def random_vector(n, seed):
    return np.random.default_rng(seed).standard_normal(n)


def c0() -> Workload:
    nx = ny = nz = 8
    mask, ubar = dirichlet(nx, ny, nz, [("x0", 0, 0.0), ("x0", 1, 0.0), ("x0", 2, 0.0)])
    return Workload("c0_le_8cube", nx, ny, nz, 1.0, 1.0, 1.0, LINEAR, 70e3, 0.3, n_steps=1,
                    mask=mask, u_bar=ubar, traction=("x1", (0.0, 0.0, -100.0)),
                    extra={"rtol": 1e-10})


def c1(n=64, n_steps=10) -> Workload:
    mask, ubar = clamp_and_compress(n, n, n, -0.1)
    return Workload(f"c1_nh_{n}cube", n, n, n, 1.0, 1.0, 1.0, NEOHOOKE, 10.0, 0.3, n_steps=n_steps,
                    mask=mask, u_bar=ubar)


def simp_patch_load(nx, ny, nz, total=(0.0, 0.0, -1.0)):
    """4x4 node patch on the x=max face, k in {0..3}, j in {ny/2-2 .. ny/2+1},
    equal share of the total force per node."""
    D = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    f = np.zeros(D)
    js = range(ny // 2 - 2, ny // 2 + 2)
    ks = range(0, 4)
    for k in ks:
        for j in js:
            n = node_index(nx, ny, nz, nx, j, k)
            f[3 * n:3 * n + 3] += np.asarray(total) / 16.0
    return f


def c2(nx=128, ny=64, nz=64, lx=2.0, ly=1.0, lz=1.0, seed=2) -> Workload:
    mask, ubar = dirichlet(nx, ny, nz, [("x0", 0, 0.0), ("x0", 1, 0.0), ("x0", 2, 0.0)])
    theta = np.random.default_rng(seed).uniform(0.01, 1.0, nx * ny * nz)
    return Workload(f"c2_simp_{nx}x{ny}x{nz}", nx, ny, nz, lx, ly, lz, SIMP, 1.0, 0.3, 3.0, 1e-3,
                    n_steps=1, mask=mask, u_bar=ubar, point_load=simp_patch_load(nx, ny, nz),
                    cell_param=theta)


def c3(n_inst=256, seed=3, lo=8, hi=32, n_steps=10):
    """List of Workloads for the batched launcher."""
    rng = np.random.default_rng(seed)
    edges = rng.integers(lo, hi + 1, n_inst)
    Es = np.exp(rng.uniform(np.log(1e2), np.log(1e4), n_inst))
    nus = rng.uniform(0.2, 0.45, n_inst)
    comp = rng.uniform(0.02, 0.15, n_inst)
    out = []
    for t in range(n_inst):
        n = int(edges[t])
        mask, ubar = clamp_and_compress(n, n, n, -float(comp[t]))
        out.append(Workload(f"c3_inst{t}_{n}cube", n, n, n, 1.0, 1.0, 1.0, NEOHOOKE, float(Es[t]),
                            float(nus[t]), n_steps=n_steps, mask=mask, u_bar=ubar))
    return out


def c4(n=128, seed=4, target_seed=5001, n_steps=5) -> Workload:
    mask, ubar = clamp_and_compress(n, n, n, -0.1)
    s = np.random.default_rng(seed).lognormal(0.0, 0.5, n * n * n)
    face = face_nodes(n, n, n, "x1")
    target = 0.02 * np.random.default_rng(target_seed).standard_normal((face.size, 3))
    return Workload(f"c4_nh_{n}cube", n, n, n, 1.0, 1.0, 1.0, NEOHOOKE, 10.0, 0.3, n_steps=n_steps,
                    mask=mask, u_bar=ubar, cell_param=s,
                    extra={"face_nodes": face, "target": target})


def fd_cells(n_cells, k=64, seed=7):
    """Cells picked for finite-difference checks."""
    return np.sort(np.random.default_rng(seed).choice(n_cells, size=min(k, n_cells), replace=False))


@dataclass
class PoissonInference:
    """Full-field inference from sparse observations (the scalar Poisson
    example): box, coefficient alpha, the boundary nodes (u = 0 there), the
    nodal source values theta_true of the bimodal source and the observed
    node ids.  One DOF per node."""
    name: str
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    alpha: float
    mask: np.ndarray        # uint8 [N], 1 = boundary node (u = 0)
    theta_true: np.ndarray  # float64 [N], nodal values of the source b
    obs: np.ndarray         # int64 [n_obs], sorted interior node ids

    @property
    def n_nodes(self):
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_cells(self):
        return self.nx * self.ny * self.nz


def boundary_nodes(nx, ny, nz):
    """uint8 [N]: 1 on every node of the six faces of the box."""
    mask = np.zeros((nx + 1) * (ny + 1) * (nz + 1), np.uint8)
    for f in ("x0", "x1", "y0", "y1", "z0", "z1"):
        mask[face_nodes(nx, ny, nz, f)] = 1
    return mask


def poisson_inference(nx=50, ny=50, nz=10, lx=1.0, ly=1.0, lz=0.2, n_obs=250, seed=11,
                      alpha=1.0) -> PoissonInference:
    """The paper's 50x50x10 hexahedra on a 1 x 1 x 0.2 box with 250 observed
    points.  Source b(x) = 10 exp(-10 |x - c1|^2) + 10 exp(-10 |x - c2|^2),
    evaluated at the nodes, with the centres c1 = (0.25 lx, 0.25 ly, 0.5 lz)
    and c2 = (0.75 lx, 0.75 ly, 0.5 lz) (the printed centres lie outside the
    box; these are their positions scaled into it).  Observed nodes: n_obs
    distinct interior nodes drawn uniformly (default_rng(seed))."""
    I, J, K = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    ids = node_index(nx, ny, nz, I, J, K).reshape(-1)
    pos = np.zeros((ids.size, 3))
    pos[ids, 0] = (lx * I / nx).reshape(-1)
    pos[ids, 1] = (ly * J / ny).reshape(-1)
    pos[ids, 2] = (lz * K / nz).reshape(-1)
    theta = np.zeros(ids.size)
    for c in ((0.25 * lx, 0.25 * ly, 0.5 * lz), (0.75 * lx, 0.75 * ly, 0.5 * lz)):
        theta += 10.0 * np.exp(-10.0 * ((pos - np.asarray(c)) ** 2).sum(axis=1))
    mask = boundary_nodes(nx, ny, nz)
    interior = np.flatnonzero(mask == 0)
    obs = np.sort(np.random.default_rng(seed).choice(interior, size=min(n_obs, interior.size),
                                                      replace=False)).astype(np.int64)
    return PoissonInference(f"poisson_{nx}x{ny}x{nz}_obs{obs.size}", nx, ny, nz, lx, ly, lz, alpha,
                            mask, theta, obs)


def j2_uniaxial(n=2, L=1.0, E=70e3, nu=0.3, sigma_y=250.0, strain_max=2.5 * 250.0 / 70e3, n_load=10,
                n_unload=10):
    """Load/unload path of the J2 plasticity example on an n^3 box of edge L:
    symmetry rollers (u_x = 0 on x=0, u_y = 0 on y=0, u_z = 0 on z=0) and
    u_z = L * strain on z=L, the strain rising from 0 to strain_max in n_load
    steps and back to 0 in n_unload steps.  Returns (mask u8[D], list of
    u_bar f64[D] per step, list of the step strains, material tuple)."""
    strains = list(np.linspace(0.0, strain_max, n_load + 1)[1:]) + \
        list(np.linspace(strain_max, 0.0, n_unload + 1)[1:])
    mask = None
    ubars = []
    for s in strains:
        mask, ub = dirichlet(n, n, n, [("x0", 0, 0.0), ("y0", 1, 0.0), ("z0", 2, 0.0), ("z1", 2, L * s)])
        ubars.append(ub)
    return mask, ubars, strains, (E, nu, sigma_y)


def topopt_cantilever(nx=16, ny=8, nz=4, lx=2.0, ly=1.0, lz=0.5, volfrac=0.5, rmin=1.5):
    """Box cantilever of the topology-optimisation loop (the paper's plate and
    bracket geometries are not available): the SIMP law of c2, x=0 clamped,
    total force (0, 0, -1) over the 4x4 node patch at the bottom of the far
    face (c2's load), volume fraction 0.5, filter radius 1.5 cells, uniform
    initial design.  Returns a Workload with extra = {volfrac, rmin}."""
    mask, ubar = dirichlet(nx, ny, nz, [("x0", 0, 0.0), ("x0", 1, 0.0), ("x0", 2, 0.0)])
    return Workload(f"topopt_cantilever_{nx}x{ny}x{nz}", nx, ny, nz, lx, ly, lz, SIMP, 1.0, 0.3, 3.0, 1e-3,
                    n_steps=1, mask=mask, u_bar=ubar, point_load=simp_patch_load(nx, ny, nz),
                    cell_param=np.full(nx * ny * nz, volfrac), extra={"volfrac": volfrac, "rmin": rmin})
