"""FP64 CPU oracle for the HEX8 weak-form path of JAX-FEM (arXiv 2212.00964).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(``paper_2212_00964_gb300``) never does.  It shares no code with the CUDA
library.

``fem_oracle.c`` holds the plain element-level definitions (shape functions,
Gauss rule, constitutive laws, element residual / JVP, assembly, the scalar
Poisson element of Sec. 3.1, the J2 return map of Sec. 2.3); this module
loads it with ctypes and exposes numpy-level functions.  ``oracle.solve``
holds the Newton / adjoint drivers (library ``spsolve`` as the linear step);
``oracle.poisson`` the forward solve, objective and adjoint gradient of the
full-field inference problem; ``oracle.plasticity`` the load-stepped J2
plasticity solve with its Gauss-point history.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fem_oracle.c")
# FEMGB_HOST_SANITIZE=1: an AddressSanitizer + UBSan build in a separate file
# (the process must run with the ASan runtime preloaded)
_SANITIZE = os.environ.get("FEMGB_HOST_SANITIZE") == "1"
_SO = os.path.join(_HERE, "liboracle_san.so" if _SANITIZE else "liboracle.so")

LINEAR, SIMP, NEOHOOKE = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile fem_oracle.c with gcc -O2 -ffp-contract=off into liboracle.so."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        san = ["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
               "-fno-sanitize-recover=all"] if _SANITIZE else ["-O2"]
        subprocess.check_call(
            ["gcc"] + san + ["-ffp-contract=off", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp,
                             "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I = ctypes.c_int
        D = ctypes.c_double
        L.oracle_shape.argtypes = [D, D, D, P, P]
        L.oracle_gauss.argtypes = [P, P]
        L.oracle_mesh.argtypes = [I, I, I, D, D, D, P, P]
        L.oracle_colour.argtypes = [I, I, I, P, P]
        L.oracle_csr_rows.argtypes = [I64, I64, P, P]
        L.oracle_csr_rows.restype = I64
        L.oracle_csr_cols.argtypes = [I64, I64, P, P, P]
        L.oracle_scatter_map.argtypes = [I64, P, P, P, P]
        L.oracle_stress.argtypes = [I, D, D, P, P]
        L.oracle_stress.restype = D
        L.oracle_dstress.argtypes = [I, D, D, P, P, P]
        mat = [I, D, D, D, D]
        L.oracle_residual.argtypes = [I64, I64, P, P] + mat + [P, P, P, P, P]
        L.oracle_residual.restype = D
        L.oracle_tangent_apply.argtypes = [I64, I64, P, P] + mat + [P, P, P, P, P]
        L.oracle_residual_mt.argtypes = [I64, P, P] + mat + [P, P, P, P, P, P, P]
        L.oracle_residual_mt.restype = D
        L.oracle_tangent_apply_mt.argtypes = [I64, P, P] + mat + [P, P, P, P, P, P, P]
        L.oracle_threads.restype = I
        L.oracle_element_tangent.argtypes = [P, P] + mat + [P, P, I64, P]
        L.oracle_diag.argtypes = [I64, I64, P, P] + mat + [P, P, P, P]
        L.oracle_assemble.argtypes = [I64, I64, P, P] + mat + [P, P, P, P, P, P, P]
        L.oracle_vjp.argtypes = [I64, I64, P, P] + mat + [P, P, P, P, P]
        L.oracle_body_force.argtypes = [I64, P, P, P, P, P]
        L.oracle_traction.argtypes = [I, I, I, P, P, I, P, P]
        L.oracle_poisson_element.argtypes = [P, P, I64, D, P, P]
        L.oracle_poisson_apply.argtypes = [I64, I64, P, P, D, P, P, P]
        L.oracle_poisson_load.argtypes = [I64, I64, P, P, P, P, P]
        L.oracle_j2_stress.argtypes = [D, D, D, P, P, P, P, P]
        L.oracle_j2_stress.restype = D
        L.oracle_j2_dstress.argtypes = [D, D, D, P, P, P, P, P]
        L.oracle_gp_jxw.argtypes = [I64, P, P, P]
        L.oracle_j2_residual.argtypes = [I64, I64, P, P, D, D, D, P, P, P, P, P, P, P, P]
        L.oracle_j2_residual.restype = I64
        L.oracle_j2_tangent_apply.argtypes = [I64, I64, P, P, D, D, D, P, P, P, P, P, P]
        L.oracle_j2_element_tangent.argtypes = [P, P, D, D, D, P, P, P, I64, P]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.uint8)


@dataclass
class Material:
    """kind: LINEAR / SIMP / NEOHOOKE; E, nu; SIMP exponent and floor."""
    kind: int
    E: float
    nu: float
    simp_p: float = 3.0
    simp_emin: float = 1e-3

    def args(self):
        return [self.kind, float(self.E), float(self.nu), float(self.simp_p), float(self.simp_emin)]


@dataclass
class Mesh:
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    conn: np.ndarray  # int32 [Ne, 8], VTK local order
    X: np.ndarray     # float64 [N, 3]

    @property
    def n_nodes(self):
        return self.X.shape[0]

    @property
    def n_cells(self):
        return self.conn.shape[0]

    @property
    def n_dofs(self):
        return 3 * self.X.shape[0]


def mesh(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0) -> Mesh:
    N = (nx + 1) * (ny + 1) * (nz + 1)
    Ne = nx * ny * nz
    conn = np.zeros((Ne, 8), np.int32)
    X = np.zeros((N, 3), np.float64)
    lib().oracle_mesh(nx, ny, nz, lx, ly, lz, _p(conn), _p(X))
    return Mesh(nx, ny, nz, lx, ly, lz, conn, X)


def with_coords(m: Mesh, X) -> Mesh:
    """Same topology, other nodal coordinates (perturbed meshes)."""
    return Mesh(m.nx, m.ny, m.nz, m.lx, m.ly, m.lz, m.conn, np.ascontiguousarray(X, np.float64))


def colour(m: Mesh):
    ptr = np.zeros(9, np.int32)
    perm = np.zeros(m.n_cells, np.int32)
    lib().oracle_colour(m.nx, m.ny, m.nz, _p(ptr), _p(perm))
    return ptr, perm


def csr(m: Mesh):
    """(row_ptr int64 [D+1], col int32 [nnz]) of the DOF graph."""
    row_ptr = np.zeros(m.n_dofs + 1, np.int64)
    nnz = lib().oracle_csr_rows(m.n_nodes, m.n_cells, _p(m.conn), _p(row_ptr))
    col = np.zeros(nnz, np.int32)
    lib().oracle_csr_cols(m.n_nodes, m.n_cells, _p(m.conn), _p(row_ptr), _p(col))
    return row_ptr, col


def scatter_map(m: Mesh, row_ptr, col):
    mp = np.zeros((m.n_cells, 24, 24), np.int32)
    lib().oracle_scatter_map(m.n_cells, _p(m.conn), _p(row_ptr), _p(col), _p(mp))
    return mp


def shape(xi, eta, zeta):
    N = np.zeros(8)
    dN = np.zeros((8, 3))
    lib().oracle_shape(xi, eta, zeta, _p(N), _p(dN))
    return N, dN


def gauss():
    gp = np.zeros((8, 3))
    w = np.zeros(8)
    lib().oracle_gauss(_p(gp), _p(w))
    return gp, w


def stress(kind, Es, nu, H):
    H = _f64(np.asarray(H).reshape(3, 3))
    P = np.zeros((3, 3))
    J = lib().oracle_stress(kind, Es, nu, _p(H), _p(P))
    return P, J


def dstress(kind, Es, nu, H, dH):
    H = _f64(np.asarray(H).reshape(3, 3))
    dH = _f64(np.asarray(dH).reshape(3, 3))
    dP = np.zeros((3, 3))
    lib().oracle_dstress(kind, Es, nu, _p(H), _p(dH), _p(dP))
    return dP


def residual(m: Mesh, mat: Material, u, cell_param=None, f_ext=None, mask=None, return_jmin=False):
    u = _f64(u).reshape(-1)
    R = np.zeros(m.n_dofs)
    cp, fe, mk = _f64(cell_param), _f64(f_ext), _u8(mask)
    jmin = lib().oracle_residual(m.n_nodes, m.n_cells, _p(m.conn), _p(m.X), *mat.args(),
                                 _p(cp), _p(u), _p(fe), _p(mk), _p(R))
    return (R, jmin) if return_jmin else R


def tangent_apply(m: Mesh, mat: Material, u, x, cell_param=None, mask=None):
    u = _f64(u).reshape(-1)
    x = _f64(x).reshape(-1)
    y = np.zeros(m.n_dofs)
    cp, mk = _f64(cell_param), _u8(mask)
    lib().oracle_tangent_apply(m.n_nodes, m.n_cells, _p(m.conn), _p(m.X), *mat.args(),
                               _p(cp), _p(u), _p(x), _p(mk), _p(y))
    return y


def threads():
    """Threads the all-cores variants run on."""
    return lib().oracle_threads()


def residual_mt(m: Mesh, mat: Material, u, cell_param=None, f_ext=None, mask=None):
    """residual() with the cell loop spread over all host cores (colour class
    by colour class); for the CPU baseline."""
    u = _f64(u).reshape(-1)
    R = np.zeros(m.n_dofs)
    cp, fe, mk = _f64(cell_param), _f64(f_ext), _u8(mask)
    ptr, perm = colour(m)
    lib().oracle_residual_mt(m.n_nodes, _p(m.conn), _p(m.X), *mat.args(), _p(cp), _p(u), _p(fe), _p(mk),
                             _p(ptr), _p(perm), _p(R))
    return R


def tangent_apply_mt(m: Mesh, mat: Material, u, x, cell_param=None, mask=None):
    """tangent_apply() with the cell loop spread over all host cores."""
    u = _f64(u).reshape(-1)
    x = _f64(x).reshape(-1)
    y = np.zeros(m.n_dofs)
    cp, mk = _f64(cell_param), _u8(mask)
    ptr, perm = colour(m)
    lib().oracle_tangent_apply_mt(m.n_nodes, _p(m.conn), _p(m.X), *mat.args(), _p(cp), _p(u), _p(x), _p(mk),
                                  _p(ptr), _p(perm), _p(y))
    return y


def element_tangent(m: Mesh, mat: Material, u, e, cell_param=None):
    u = _f64(u).reshape(-1)
    Ke = np.zeros((24, 24))
    cp = _f64(cell_param)
    lib().oracle_element_tangent(_p(m.conn), _p(m.X), *mat.args(), _p(cp), _p(u), int(e), _p(Ke))
    return Ke


def diag(m: Mesh, mat: Material, u, cell_param=None, mask=None):
    u = _f64(u).reshape(-1)
    d = np.zeros(m.n_dofs)
    cp, mk = _f64(cell_param), _u8(mask)
    lib().oracle_diag(m.n_nodes, m.n_cells, _p(m.conn), _p(m.X), *mat.args(), _p(cp), _p(u),
                      _p(mk), _p(d))
    return d


def assemble_vals(m: Mesh, mat: Material, u, row_ptr, col, smap, cell_param=None, mask=None):
    u = _f64(u).reshape(-1)
    vals = np.zeros(len(col))
    cp, mk = _f64(cell_param), _u8(mask)
    lib().oracle_assemble(m.n_nodes, m.n_cells, _p(m.conn), _p(m.X), *mat.args(), _p(cp), _p(u),
                          _p(mk), _p(np.ascontiguousarray(row_ptr, np.int64)),
                          _p(np.ascontiguousarray(col, np.int32)),
                          _p(np.ascontiguousarray(smap, np.int32)), _p(vals))
    return vals


def assemble(m: Mesh, mat: Material, u, cell_param=None, mask=None, pattern=None):
    """Global K(u) as a scipy CSR matrix (Algorithm 1)."""
    import scipy.sparse as sp
    if pattern is None:
        row_ptr, col = csr(m)
        pattern = (row_ptr, col, scatter_map(m, row_ptr, col))
    row_ptr, col, smap = pattern
    vals = assemble_vals(m, mat, u, row_ptr, col, smap, cell_param, mask)
    return sp.csr_matrix((vals, col, row_ptr), shape=(m.n_dofs, m.n_dofs))


def vjp(m: Mesh, mat: Material, u, lam, cell_param=None, mask=None):
    u = _f64(u).reshape(-1)
    lam = _f64(lam).reshape(-1)
    g = np.zeros(m.n_cells)
    cp, mk = _f64(cell_param), _u8(mask)
    lib().oracle_vjp(m.n_nodes, m.n_cells, _p(m.conn), _p(m.X), *mat.args(), _p(cp), _p(u),
                     _p(lam), _p(mk), _p(g))
    return g


def gauss_points_phys(m: Mesh):
    xg = np.zeros((m.n_cells, 8, 3))
    lib().oracle_body_force(m.n_cells, _p(m.conn), _p(m.X), None, None, _p(xg))
    return xg


def body_force(m: Mesh, b_gp):
    b = _f64(np.asarray(b_gp).reshape(m.n_cells, 8, 3))
    f = np.zeros(m.n_dofs)
    lib().oracle_body_force(m.n_cells, _p(m.conn), _p(m.X), _p(b), _p(f), None)
    return f


FACES = {"x0": 0, "x1": 1, "y0": 2, "y1": 3, "z0": 4, "z1": 5}


def traction(m: Mesh, face, t):
    f = np.zeros(m.n_dofs)
    t = _f64(np.asarray(t, np.float64).reshape(3))
    fid = FACES[face] if isinstance(face, str) else int(face)
    lib().oracle_traction(m.nx, m.ny, m.nz, _p(m.conn), _p(m.X), fid, _p(t), _p(f))
    return f
