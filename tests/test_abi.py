"""CPU checks of the C-ABI boundary: the library builds, loads without a GPU
and exports every entry point that include/fem.h declares; status strings
and option defaults are host-only and callable here."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    hdr = open(os.path.join(ROOT, "include", "fem.h")).read()
    return re.findall(r"^\s*(?:int|void|const char \*|int64_t)\s*\**\s*(fem_\w+)\s*\(", hdr, re.M)


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for n in ["fem_mesh", "fem_residual", "fem_tangent_apply", "fem_solve", "fem_adjoint",
              "fem_solve_batched", "fem_vjp", "fem_tangent_diag", "fem_assemble_csr"]:
        assert n in names


def test_library_loads_and_exports_every_symbol():
    from paper_2212_00964_gb300 import build
    so = build.build()
    L = ctypes.CDLL(so)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_host_only_calls():
    from paper_2212_00964_gb300 import build, fem
    build.build()
    L = fem.lib()
    assert L.fem_status_string(fem.FEM_ERR_INVERTED).decode().startswith("inverted")
    o = fem.default_options()
    assert o.precision == fem.FEM_MIXED and o.newton_maxit > 0 and 0 < o.pcg_rtol < 1
    # argument validation happens on the host, before any CUDA call
    h = ctypes.c_void_p()
    assert L.fem_mesh(0, 1, 1, 1.0, 1.0, 1.0, 0, None, ctypes.byref(h)) == fem.FEM_ERR_ARG
    assert L.fem_mesh(2, 2, 2, -1.0, 1.0, 1.0, 0, None, ctypes.byref(h)) == fem.FEM_ERR_ARG
    assert L.fem_mesh(2, 2, 2, 1.0, 1.0, 1.0, 0, None, None) == fem.FEM_ERR_ARG
    assert "NULL" in L.fem_last_error().decode() or "out" in L.fem_last_error().decode()
    mat = fem.material(7, 1.0, 0.3)
    assert L.fem_residual(None, ctypes.byref(mat), 0, None, None, None, None, None, None) == fem.FEM_ERR_ARG
