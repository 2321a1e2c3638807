"""Thin Python binding of the C-ABI in include/fem.h (argument marshalling only).

Every function has the name of the C entry point it calls.  Arrays are torch
CUDA tensors (device memory and the current stream come from PyTorch); every
computation runs in libfemgb.so.  If the library is missing the binding
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_lib", "libfemgb.so")

FEM_OK = 0
FEM_ERR_ARG, FEM_ERR_CUDA, FEM_ERR_NOT_CONVERGED, FEM_ERR_INVERTED = -1, -2, -3, -4
FEM_ERR_BREAKDOWN, FEM_ERR_NONFINITE, FEM_ERR_TIMEOUT, FEM_ERR_NOMEM = -5, -6, -7, -8
FEM_LINEAR, FEM_SIMP, FEM_NEOHOOKE = 0, 1, 2
FEM_FP64, FEM_FP32, FEM_MIXED = 0, 1, 2
FEM_MESH_CSR = 1
FEM_MESH_DETERMINISTIC = 2
FEM_MESH_TENSOR_CORES = 4
FEM_POISSON_STIFFNESS, FEM_POISSON_MASS = 0, 1
FACES = {"x0": 0, "x1": 1, "y0": 2, "y1": 3, "z0": 4, "z1": 5}


class FemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class fem_material(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("E", ctypes.c_double), ("nu", ctypes.c_double),
                ("simp_p", ctypes.c_double), ("simp_emin", ctypes.c_double)]


class fem_j2_material(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("nu", ctypes.c_double), ("sigma_y", ctypes.c_double)]


class fem_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("newton_rtol", ctypes.c_double),
                ("newton_atol", ctypes.c_double), ("newton_maxit", ctypes.c_int),
                ("pcg_rtol", ctypes.c_double), ("pcg_maxit", ctypes.c_int),
                ("pcg_chunk", ctypes.c_int), ("step_begin", ctypes.c_int),
                ("apply_kernel", ctypes.c_int), ("cg_fused", ctypes.c_int),
                ("timeout_s", ctypes.c_double), ("newton_res32", ctypes.c_int), ("graph_loop", ctypes.c_int),
                ("pcg_rtol_max", ctypes.c_double), ("cta_cells", ctypes.c_int)]


class fem_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("load_steps", ctypes.c_int), ("newton_iters", ctypes.c_int),
                ("pcg_iters", ctypes.c_int), ("ref_rnorm", ctypes.c_double),
                ("final_rnorm", ctypes.c_double), ("time_ms", ctypes.c_double),
                ("apply_ms", ctypes.c_double), ("apply_samples", ctypes.c_int), ("apply_launches", ctypes.c_int),
                ("apply_kernel", ctypes.c_int), ("update_ms", ctypes.c_double), ("update_samples", ctypes.c_int),
                ("cta_cells", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class fem_bc(ctypes.Structure):
    _fields_ = [("mask", ctypes.c_void_p), ("u_bar", ctypes.c_void_p), ("f_ext", ctypes.c_void_p)]


class fem_instance(ctypes.Structure):
    _fields_ = [("mesh", ctypes.c_void_p), ("mat", fem_material), ("bc", fem_bc),
                ("cell_param", ctypes.c_void_p), ("n_steps", ctypes.c_int), ("u_inout", ctypes.c_void_p)]


_lib = None


def lib():
    """Load libfemgb.so (built by ``paper_2212_00964_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_SO):
        raise RuntimeError(f"{_SO} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(_SO)
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    MP = ctypes.POINTER(fem_material)
    L.fem_mesh.argtypes = [I, I, I, D, D, D, I, P, ctypes.POINTER(P)]
    L.fem_mesh_info.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]
    L.fem_mesh_export.argtypes = [P] * 8 + [P]
    L.fem_mesh_destroy.argtypes = [P]
    L.fem_load_traction.argtypes = [P, I, P, P, P]
    L.fem_load_body.argtypes = [P, P, P, P]
    L.fem_residual.argtypes = [P, MP, I, P, P, P, P, P, P]
    L.fem_tangent_apply.argtypes = [P, MP, I, P, P, P, P, P, P]
    L.fem_tangent_diag.argtypes = [P, MP, I, P, P, P, P, P]
    L.fem_vjp.argtypes = [P, MP, I, P, P, P, P, P, P]
    L.fem_assemble_csr.argtypes = [P, MP, I, P, P, P, P, P]
    L.fem_bicgstab_csr.argtypes = [P, I, P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D), P]
    JP = ctypes.POINTER(fem_j2_material)
    L.fem_j2_residual.argtypes = [P, JP, P, P, P, P, P, ctypes.POINTER(I64), P]
    L.fem_j2_tangent_apply.argtypes = [P, JP, I, P, P, P, P, P, P]
    L.fem_j2_step.argtypes = [P, JP, I, P, P, P, P, D, I, D, I, ctypes.POINTER(I), ctypes.POINTER(I),
                              ctypes.POINTER(I64), P]
    L.fem_density_filter.argtypes = [P, D, I, P, P, P]
    L.fem_oc_step.argtypes = [P, P, P, P, D, D, D, D, P, ctypes.POINTER(D), P]
    L.fem_mma_step.argtypes = [P, P, D, P, P, D, D, I, P, P, P, P, P, ctypes.POINTER(D), P]
    L.fem_poisson_adjoint.argtypes = [P, I, D, P, P, D, I, P, P, ctypes.POINTER(I), P]
    L.fem_poisson_apply.argtypes = [P, I, D, I, P, P, P, P]
    L.fem_poisson_solve.argtypes = [P, I, D, P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D), P]
    L.fem_poisson_gradient.argtypes = [P, I, D, P, P, P, P, I64, D, I, P, P, P, ctypes.POINTER(D),
                                       ctypes.POINTER(I), P]
    L.fem_default_options.argtypes = [ctypes.POINTER(fem_options)]
    L.fem_default_options.restype = None
    L.fem_solve.argtypes = [P, MP, ctypes.POINTER(fem_bc), P, I, ctypes.POINTER(fem_options), P,
                            ctypes.POINTER(fem_stats), P]
    L.fem_adjoint.argtypes = [P, MP, ctypes.POINTER(fem_bc), P, P, P, P, ctypes.POINTER(fem_options),
                              P, P, ctypes.POINTER(fem_stats), P]
    L.fem_solve_batched.argtypes = [I, ctypes.POINTER(fem_instance), ctypes.POINTER(fem_options),
                                    ctypes.POINTER(fem_stats), P]
    L.fem_solve_static.argtypes = [I, I, I, D, D, D, MP, ctypes.POINTER(fem_bc), P, I,
                                   ctypes.POINTER(fem_options), P, ctypes.POINTER(fem_stats), P]
    L.fem_status_string.argtypes = [I]
    L.fem_status_string.restype = ctypes.c_char_p
    L.fem_last_error.restype = ctypes.c_char_p
    L.fem_kernel_launches.restype = I64
    _lib = L
    return L


def _check(rc, what):
    if rc != FEM_OK:
        L = lib()
        raise FemError(rc, f"{what}: {L.fem_status_string(rc).decode()}: {L.fem_last_error().decode()}")
    return rc


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor], dtype=None, n=None, name="array"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def kernel_launches() -> int:
    return int(lib().fem_kernel_launches())


def material(kind, E, nu, simp_p=3.0, simp_emin=1e-3) -> fem_material:
    return fem_material(int(kind), float(E), float(nu), float(simp_p), float(simp_emin))


def default_options(**kw) -> fem_options:
    o = fem_options()
    lib().fem_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Mesh:
    """Owner of a fem_mesh_t handle."""

    def __init__(self, handle, nx, ny, nz, lx, ly, lz, csr):
        self.handle = handle
        self.nx, self.ny, self.nz = nx, ny, nz
        self.lx, self.ly, self.lz = lx, ly, lz
        self.csr = csr
        n = ctypes.c_int64()
        e = ctypes.c_int64()
        z = ctypes.c_int64()
        _check(lib().fem_mesh_info(handle, ctypes.byref(n), ctypes.byref(e), ctypes.byref(z)), "fem_mesh_info")
        self.n_nodes, self.n_cells, self.nnz = n.value, e.value, z.value

    @property
    def n_dofs(self):
        return 3 * self.n_nodes

    def close(self):
        if self.handle:
            lib().fem_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fem_mesh(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, csr=False, stream=None, deterministic=False,
             tensor_cores=False) -> Mesh:
    h = ctypes.c_void_p()
    flags = ((FEM_MESH_CSR if csr else 0) | (FEM_MESH_DETERMINISTIC if deterministic else 0)
             | (FEM_MESH_TENSOR_CORES if tensor_cores else 0))
    _check(lib().fem_mesh(nx, ny, nz, lx, ly, lz, flags, _stream(stream), ctypes.byref(h)), "fem_mesh")
    return Mesh(h, nx, ny, nz, lx, ly, lz, csr)


def fem_mesh_export(m: Mesh, stream=None, csr=False):
    dev = torch.device("cuda")
    out = {
        "conn": torch.empty((m.n_cells, 8), dtype=torch.int32, device=dev),
        "X": torch.empty((m.n_nodes, 3), dtype=torch.float64, device=dev),
        "colour_ptr": torch.empty(9, dtype=torch.int32, device=dev),
        "cell_perm": torch.empty(m.n_cells, dtype=torch.int32, device=dev),
    }
    if csr:
        out["row_ptr"] = torch.empty(m.n_dofs + 1, dtype=torch.int32, device=dev)
        out["col"] = torch.empty(m.nnz, dtype=torch.int32, device=dev)
        out["map"] = torch.empty((m.n_cells, 24, 24), dtype=torch.int32, device=dev)
    g = lambda k: _ptr(out.get(k))
    _check(lib().fem_mesh_export(m.handle, g("conn"), g("X"), g("colour_ptr"), g("cell_perm"), g("row_ptr"),
                                 g("col"), g("map"), _stream(stream)), "fem_mesh_export")
    return out


def fem_load_traction(m: Mesh, face, t, f_ext: torch.Tensor, stream=None):
    tt = (ctypes.c_double * 3)(*[float(v) for v in t])
    fid = FACES[face] if isinstance(face, str) else int(face)
    _check(lib().fem_load_traction(m.handle, fid, tt, _ptr(f_ext, torch.float64, m.n_dofs, "f_ext"),
                                   _stream(stream)), "fem_load_traction")
    return f_ext


def fem_load_body(m: Mesh, b, f_ext: torch.Tensor, stream=None):
    bb = (ctypes.c_double * 3)(*[float(v) for v in b])
    _check(lib().fem_load_body(m.handle, bb, _ptr(f_ext, torch.float64, m.n_dofs, "f_ext"), _stream(stream)),
           "fem_load_body")
    return f_ext


def _prec(dtype):
    if dtype == torch.float64:
        return FEM_FP64
    if dtype == torch.float32:
        return FEM_FP32
    raise TypeError("cell operators take float64 or float32 tensors")


def fem_residual(m: Mesh, mat: fem_material, u, cell_param=None, mask=None, f_ext=None, r=None, stream=None):
    dt = u.dtype
    r = torch.empty_like(u) if r is None else r
    _check(lib().fem_residual(m.handle, ctypes.byref(mat), _prec(dt), _ptr(u, dt, m.n_dofs, "u"),
                              _ptr(cell_param, dt, m.n_cells, "cell_param"),
                              _ptr(mask, torch.uint8, m.n_dofs, "mask"), _ptr(f_ext, dt, m.n_dofs, "f_ext"),
                              _ptr(r, dt, m.n_dofs, "r"), _stream(stream)), "fem_residual")
    return r


def fem_tangent_apply(m: Mesh, mat: fem_material, u, x, cell_param=None, mask=None, y=None, stream=None):
    dt = u.dtype
    y = torch.empty_like(x) if y is None else y
    _check(lib().fem_tangent_apply(m.handle, ctypes.byref(mat), _prec(dt), _ptr(u, dt, m.n_dofs, "u"),
                                   _ptr(cell_param, dt, m.n_cells, "cell_param"),
                                   _ptr(mask, torch.uint8, m.n_dofs, "mask"), _ptr(x, dt, m.n_dofs, "x"),
                                   _ptr(y, dt, m.n_dofs, "y"), _stream(stream)), "fem_tangent_apply")
    return y


def fem_tangent_diag(m: Mesh, mat: fem_material, u, cell_param=None, mask=None, d=None, stream=None):
    dt = u.dtype
    d = torch.empty_like(u) if d is None else d
    _check(lib().fem_tangent_diag(m.handle, ctypes.byref(mat), _prec(dt), _ptr(u, dt, m.n_dofs, "u"),
                                  _ptr(cell_param, dt, m.n_cells, "cell_param"),
                                  _ptr(mask, torch.uint8, m.n_dofs, "mask"), _ptr(d, dt, m.n_dofs, "d"),
                                  _stream(stream)), "fem_tangent_diag")
    return d


def fem_vjp(m: Mesh, mat: fem_material, u, lam, cell_param=None, mask=None, g=None, stream=None):
    dt = u.dtype
    g = torch.empty(m.n_cells, dtype=dt, device=u.device) if g is None else g
    _check(lib().fem_vjp(m.handle, ctypes.byref(mat), _prec(dt), _ptr(u, dt, m.n_dofs, "u"),
                         _ptr(lam, dt, m.n_dofs, "lambda"), _ptr(cell_param, dt, m.n_cells, "cell_param"),
                         _ptr(mask, torch.uint8, m.n_dofs, "mask"), _ptr(g, dt, m.n_cells, "g"),
                         _stream(stream)), "fem_vjp")
    return g


def fem_assemble_csr(m: Mesh, mat: fem_material, u, cell_param=None, mask=None, vals=None, stream=None):
    dt = u.dtype
    vals = torch.empty(m.nnz, dtype=dt, device=u.device) if vals is None else vals
    _check(lib().fem_assemble_csr(m.handle, ctypes.byref(mat), _prec(dt), _ptr(u, dt, m.n_dofs, "u"),
                                  _ptr(cell_param, dt, m.n_cells, "cell_param"),
                                  _ptr(mask, torch.uint8, m.n_dofs, "mask"), _ptr(vals, dt, m.nnz, "vals"),
                                  _stream(stream)), "fem_assemble_csr")
    return vals


def fem_bicgstab_csr(m: Mesh, vals, b, x=None, rtol=1e-10, maxit=10000, stream=None, check=True):
    """Jacobi-BiCGSTAB on an assembled matrix; returns (x, iterations, ||r||/||b||)."""
    dt = vals.dtype
    x = torch.zeros_like(b) if x is None else x
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    rc = lib().fem_bicgstab_csr(m.handle, _prec(dt), _ptr(vals, dt, m.nnz, "vals"), _ptr(b, dt, m.n_dofs, "b"),
                                _ptr(x, dt, m.n_dofs, "x"), ctypes.c_double(rtol), int(maxit), ctypes.byref(it),
                                ctypes.byref(res), _stream(stream))
    if check:
        _check(rc, "fem_bicgstab_csr")
    return x, it.value, res.value


def fem_poisson_apply(m: Mesh, x, alpha=1.0, op=FEM_POISSON_STIFFNESS, mask=None, y=None, stream=None):
    """y = A x (stiffness, prescribed columns removed, y_c = x_c) or y = M x
    (mass, y_c = 0) of the scalar Poisson problem; per-node arrays."""
    dt = x.dtype
    y = torch.empty_like(x) if y is None else y
    _check(lib().fem_poisson_apply(m.handle, _prec(dt), ctypes.c_double(alpha), int(op),
                                   _ptr(mask, torch.uint8, m.n_nodes, "mask"), _ptr(x, dt, m.n_nodes, "x"),
                                   _ptr(y, dt, m.n_nodes, "y"), _stream(stream)), "fem_poisson_apply")
    return y


def _poisson_prec(dt, mixed):
    if mixed:
        if dt != torch.float64:
            raise TypeError("the mixed-precision Poisson calls take float64 tensors")
        return FEM_MIXED
    return _prec(dt)


def _poisson_rtol(rtol, dt, mixed):
    # FP32 CG stalls near 1e-7 relative, so its default is looser
    if rtol is not None:
        return rtol
    return 1e-6 if (dt == torch.float32 and not mixed) else 1e-10


def fem_poisson_solve(m: Mesh, b, alpha=1.0, mask=None, u=None, rtol=None, maxit=10000, stream=None,
                      check=True, mixed=False):
    """Jacobi-PCG for the eliminated Poisson stiffness (mixed=True: FP32 CG
    under FP64 refinement): returns (u, iterations, ||r||/||b||).  rtol
    defaults to 1e-10 (FP64, mixed) or 1e-6 (FP32)."""
    dt = b.dtype
    rtol = _poisson_rtol(rtol, dt, mixed)
    u = torch.zeros_like(b) if u is None else u
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    rc = lib().fem_poisson_solve(m.handle, _poisson_prec(dt, mixed), ctypes.c_double(alpha),
                                 _ptr(mask, torch.uint8, m.n_nodes, "mask"), _ptr(b, dt, m.n_nodes, "b"),
                                 _ptr(u, dt, m.n_nodes, "u"), ctypes.c_double(rtol), int(maxit), ctypes.byref(it),
                                 ctypes.byref(res), _stream(stream))
    if check:
        _check(rc, "fem_poisson_solve")
    return u, it.value, res.value


def fem_poisson_adjoint(m: Mesh, dJdu, alpha=1.0, mask=None, rtol=None, maxit=10000, stream=None, mixed=False):
    """(du/dtheta)^T dJdu for theta -> u(theta) (A u = M theta): returns (grad, lambda, iterations)."""
    dt = dJdu.dtype
    rtol = _poisson_rtol(rtol, dt, mixed)
    lam = torch.empty_like(dJdu)
    grad = torch.empty_like(dJdu)
    it = ctypes.c_int(0)
    _check(lib().fem_poisson_adjoint(m.handle, _poisson_prec(dt, mixed), ctypes.c_double(alpha),
                                     _ptr(mask, torch.uint8, m.n_nodes, "mask"), _ptr(dJdu, dt, m.n_nodes, "dJdu"),
                                     ctypes.c_double(rtol), int(maxit), _ptr(lam, dt, m.n_nodes, "lambda"),
                                     _ptr(grad, dt, m.n_nodes, "grad"), ctypes.byref(it), _stream(stream)),
           "fem_poisson_adjoint")
    return grad, lam, it.value


def fem_poisson_gradient(m: Mesh, theta, obs, u_obs, alpha=1.0, mask=None, rtol=None, maxit=10000,
                         stream=None, mixed=False):
    """Objective of the full-field inference problem and its adjoint
    gradient: returns dict(J, grad, u, lam, iters)."""
    dt = theta.dtype
    rtol = _poisson_rtol(rtol, dt, mixed)
    prec = _poisson_prec(dt, mixed)
    u = torch.empty_like(theta)
    lam = torch.empty_like(theta)
    grad = torch.empty_like(theta)
    J = ctypes.c_double(0.0)
    its = (ctypes.c_int * 2)()
    n_obs = obs.numel()
    _check(lib().fem_poisson_gradient(m.handle, prec, ctypes.c_double(alpha),
                                      _ptr(mask, torch.uint8, m.n_nodes, "mask"),
                                      _ptr(theta, dt, m.n_nodes, "theta"), _ptr(obs, torch.int64, n_obs, "obs"),
                                      _ptr(u_obs, dt, n_obs, "u_obs"), int(n_obs), ctypes.c_double(rtol),
                                      int(maxit), _ptr(u, dt, m.n_nodes, "u"), _ptr(lam, dt, m.n_nodes, "lam"),
                                      _ptr(grad, dt, m.n_nodes, "grad"), ctypes.byref(J), its,
                                      _stream(stream)), "fem_poisson_gradient")
    return {"J": J.value, "grad": grad, "u": u, "lam": lam, "iters": (its[0], its[1])}


def fem_density_filter(m: Mesh, g, rmin=1.5, out=None, stream=None, transpose=False):
    """Cone-kernel filter over the cells (float64 [n_cells]); transpose=True
    applies its transpose (the chain rule of a filtered density)."""
    out = torch.empty_like(g) if out is None else out
    _check(lib().fem_density_filter(m.handle, ctypes.c_double(rmin), int(bool(transpose)),
                                     _ptr(g, torch.float64, m.n_cells, "g"),
                                     _ptr(out, torch.float64, m.n_cells, "out"), _stream(stream)),
           "fem_density_filter")
    return out


def fem_oc_step(m: Mesh, x, g, dv, volfrac, move=0.2, x_min=0.0, x_max=1.0, stream=None):
    """Optimality-criteria update; returns (y, lam)."""
    n = m.n_cells
    y = torch.empty_like(x)
    lam = ctypes.c_double(0.0)
    _check(lib().fem_oc_step(m.handle, _ptr(x, torch.float64, n, "x"), _ptr(g, torch.float64, n, "g"),
                             _ptr(dv, torch.float64, n, "dv"), ctypes.c_double(volfrac), ctypes.c_double(move),
                             ctypes.c_double(x_min), ctypes.c_double(x_max), _ptr(y, torch.float64, n, "y"),
                             ctypes.byref(lam), _stream(stream)), "fem_oc_step")
    return y, lam.value


class MMAState:
    """Caller-owned state of fem_mma_step (device arrays [n_cells])."""

    def __init__(self, m: Mesh, x_min=0.0, x_max=1.0):
        z = lambda: torch.zeros(m.n_cells, dtype=torch.float64, device="cuda")
        self.m, self.x_min, self.x_max = m, float(x_min), float(x_max)
        self.x1, self.x2, self.low, self.upp = z(), z(), z(), z()
        self.iter = 0
        self.lam = 0.0

    def step(self, x, f1, df0, df1, stream=None):
        n = self.m.n_cells
        y = torch.empty_like(x)
        lam = ctypes.c_double(0.0)
        _check(lib().fem_mma_step(self.m.handle, _ptr(x, torch.float64, n, "x"), ctypes.c_double(f1),
                                  _ptr(df0, torch.float64, n, "df0"), _ptr(df1, torch.float64, n, "df1"),
                                  ctypes.c_double(self.x_min), ctypes.c_double(self.x_max), int(self.iter),
                                  _ptr(self.x1, torch.float64, n), _ptr(self.x2, torch.float64, n),
                                  _ptr(self.low, torch.float64, n), _ptr(self.upp, torch.float64, n),
                                  _ptr(y, torch.float64, n, "y"), ctypes.byref(lam), _stream(stream)),
               "fem_mma_step")
        self.iter += 1
        self.lam = lam.value
        return y


def j2_material(E, nu, sigma_y) -> fem_j2_material:
    return fem_j2_material(float(E), float(nu), float(sigma_y))


def j2_history(m: Mesh):
    """Virgin Gauss-point history (float64 [12 * 8 * n_cells], all zeros)."""
    return torch.zeros(12 * 8 * m.n_cells, dtype=torch.float64, device="cuda")


def fem_j2_residual(m: Mesh, mat: fem_j2_material, u, hist, mask=None, r=None, hist_new=None, stream=None):
    """(r, n_yield) of perfect J2 plasticity; hist_new (if given) receives
    the returned states."""
    H = 12 * 8 * m.n_cells
    r = torch.empty_like(u) if r is None else r
    ny = ctypes.c_int64(0)
    _check(lib().fem_j2_residual(m.handle, ctypes.byref(mat), _ptr(mask, torch.uint8, m.n_dofs, "mask"),
                                 _ptr(u, torch.float64, m.n_dofs, "u"), _ptr(hist, torch.float64, H, "hist"),
                                 _ptr(r, torch.float64, m.n_dofs, "r"),
                                 _ptr(hist_new, torch.float64, H, "hist_new"), ctypes.byref(ny), _stream(stream)),
           "fem_j2_residual")
    return r, ny.value


def fem_j2_tangent_apply(m: Mesh, mat: fem_j2_material, u, hist, x, mask=None, y=None, stream=None):
    """y = K(u) x; x float64 (FP64) or float32 (FP32 from the FP64 state)."""
    H = 12 * 8 * m.n_cells
    dt = x.dtype
    y = torch.empty_like(x) if y is None else y
    _check(lib().fem_j2_tangent_apply(m.handle, ctypes.byref(mat), _prec(dt),
                                      _ptr(mask, torch.uint8, m.n_dofs, "mask"),
                                      _ptr(u, torch.float64, m.n_dofs, "u"), _ptr(hist, torch.float64, H, "hist"),
                                      _ptr(x, dt, m.n_dofs, "x"), _ptr(y, dt, m.n_dofs, "y"),
                                      _stream(stream)), "fem_j2_tangent_apply")
    return y


def fem_j2_step(m: Mesh, mat: fem_j2_material, mask, u_bar, u, hist, newton_rtol=1e-10, newton_maxit=30,
                cg_rtol=None, cg_maxit=20000, stream=None, mixed=False):
    """One load step in place (u, hist); mixed=True: FP32 tangent and CG
    inside the FP64 Newton.  Returns dict(newton_iters, cg_iters, n_yield)."""
    H = 12 * 8 * m.n_cells
    if cg_rtol is None:
        cg_rtol = 1e-4 if mixed else 1e-10
    ni, ci, ny = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int64(0)
    _check(lib().fem_j2_step(m.handle, ctypes.byref(mat), FEM_MIXED if mixed else FEM_FP64,
                             _ptr(mask, torch.uint8, m.n_dofs, "mask"),
                             _ptr(u_bar, torch.float64, m.n_dofs, "u_bar"), _ptr(u, torch.float64, m.n_dofs, "u"),
                             _ptr(hist, torch.float64, H, "hist"), ctypes.c_double(newton_rtol), int(newton_maxit),
                             ctypes.c_double(cg_rtol), int(cg_maxit), ctypes.byref(ni), ctypes.byref(ci),
                             ctypes.byref(ny), _stream(stream)), "fem_j2_step")
    return {"newton_iters": ni.value, "cg_iters": ci.value, "n_yield": ny.value}


def _bc(m: Mesh, mask, u_bar=None, f_ext=None) -> fem_bc:
    return fem_bc(_ptr(mask, torch.uint8, m.n_dofs, "mask"), _ptr(u_bar, torch.float64, m.n_dofs, "u_bar"),
                  _ptr(f_ext, torch.float64, m.n_dofs, "f_ext"))


def fem_solve(m: Mesh, mat: fem_material, mask, u_bar, u, f_ext=None, cell_param=None, n_steps=1,
              options: Optional[fem_options] = None, stream=None, check=True):
    """Solve in place into u (float64 [D]); returns the fem_stats as a dict."""
    bc = _bc(m, mask, u_bar, f_ext)
    st = fem_stats()
    rc = lib().fem_solve(m.handle, ctypes.byref(mat), ctypes.byref(bc),
                         _ptr(cell_param, torch.float64, m.n_cells, "cell_param"), int(n_steps),
                         ctypes.byref(options) if options is not None else None,
                         _ptr(u, torch.float64, m.n_dofs, "u"), ctypes.byref(st), _stream(stream))
    if check:
        _check(rc, "fem_solve")
    d = st.as_dict()
    d["rc"] = rc
    return d


def fem_adjoint(m: Mesh, mat: fem_material, mask, u_star, dJdu, cell_param=None, dJdtheta_explicit=None,
                options: Optional[fem_options] = None, lam=None, stream=None, check=True):
    """Returns (dJ/dtheta [Ne] float64, stats dict)."""
    g = torch.empty(m.n_cells, dtype=torch.float64, device=u_star.device)
    bc = _bc(m, mask)
    st = fem_stats()
    rc = lib().fem_adjoint(m.handle, ctypes.byref(mat), ctypes.byref(bc),
                           _ptr(u_star, torch.float64, m.n_dofs, "u_star"),
                           _ptr(cell_param, torch.float64, m.n_cells, "cell_param"),
                           _ptr(dJdu, torch.float64, m.n_dofs, "dJdu"),
                           _ptr(dJdtheta_explicit, torch.float64, m.n_cells, "dJdtheta_explicit"),
                           ctypes.byref(options) if options is not None else None,
                           _ptr(g, torch.float64, m.n_cells, "dJdtheta_out"),
                           _ptr(lam, torch.float64, m.n_dofs, "lambda_out"), ctypes.byref(st), _stream(stream))
    if check:
        _check(rc, "fem_adjoint")
    d = st.as_dict()
    d["rc"] = rc
    return g, d


def fem_solve_static(nx, ny, nz, lx, ly, lz, mat: fem_material, mask, u_bar, u, f_ext=None, cell_param=None,
                     n_steps=1, options: Optional[fem_options] = None, stream=None, check=True):
    """fem_solve for one box without a mesh handle or any device allocation:
    scratch comes from the library's fixed static device array (see
    include/fem.h for the size limit and the sharing rules)."""
    D = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    bc = fem_bc(_ptr(mask, torch.uint8, D, "mask"), _ptr(u_bar, torch.float64, D, "u_bar"),
                _ptr(f_ext, torch.float64, D, "f_ext"))
    st = fem_stats()
    rc = lib().fem_solve_static(int(nx), int(ny), int(nz), float(lx), float(ly), float(lz), ctypes.byref(mat),
                                ctypes.byref(bc), _ptr(cell_param, torch.float64, nx * ny * nz, "cell_param"),
                                int(n_steps), ctypes.byref(options) if options is not None else None,
                                _ptr(u, torch.float64, D, "u"), ctypes.byref(st), _stream(stream))
    if check:
        _check(rc, "fem_solve_static")
    d = st.as_dict()
    d["rc"] = rc
    return d


@dataclass
class Instance:
    mesh: Mesh
    mat: fem_material
    mask: torch.Tensor
    u_bar: torch.Tensor
    u: torch.Tensor
    n_steps: int = 1
    f_ext: Optional[torch.Tensor] = None
    cell_param: Optional[torch.Tensor] = None


def fem_solve_batched(instances: Sequence[Instance], options: Optional[fem_options] = None, stream=None,
                      check=True):
    n = len(instances)
    arr = (fem_instance * n)()
    for k, I in enumerate(instances):
        m = I.mesh
        arr[k].mesh = m.handle
        arr[k].mat = I.mat
        arr[k].bc = _bc(m, I.mask, I.u_bar, I.f_ext)
        arr[k].cell_param = _ptr(I.cell_param, torch.float64, m.n_cells, "cell_param")
        arr[k].n_steps = int(I.n_steps)
        arr[k].u_inout = _ptr(I.u, torch.float64, m.n_dofs, "u")
    stats = (fem_stats * n)()
    rc = lib().fem_solve_batched(n, arr, ctypes.byref(options) if options is not None else None, stats,
                                 _stream(stream))
    if check:
        _check(rc, "fem_solve_batched")
    return rc, [s.as_dict() for s in stats]
