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
    # the scalar Poisson entry points validate on the host too
    assert L.fem_poisson_apply(None, 0, 1.0, 0, None, None, None, None) == fem.FEM_ERR_ARG
    assert L.fem_poisson_solve(None, 0, 1.0, None, None, None, 1e-8, 10, None, None, None) == fem.FEM_ERR_ARG
    assert L.fem_poisson_gradient(None, 0, 1.0, None, None, None, None, 0, 1e-8, 10, None, None, None, None,
                                  None, None) == fem.FEM_ERR_ARG
    assert L.fem_poisson_adjoint(None, 0, 1.0, None, None, 1e-8, 10, None, None, None, None) == fem.FEM_ERR_ARG
    assert "NULL mesh" in L.fem_last_error().decode()
    jm = fem.j2_material(70e3, 0.3, 250.0)
    assert L.fem_j2_residual(None, ctypes.byref(jm), None, None, None, None, None, None, None) == fem.FEM_ERR_ARG
    assert L.fem_j2_tangent_apply(None, ctypes.byref(jm), 0, None, None, None, None, None, None) == fem.FEM_ERR_ARG
    assert L.fem_j2_step(None, ctypes.byref(jm), 0, None, None, None, None, 1e-10, 10, 1e-10, 10, None, None,
                         None, None) == fem.FEM_ERR_ARG
    assert L.fem_density_filter(None, 1.5, 0, None, None, None) == fem.FEM_ERR_ARG
    assert L.fem_oc_step(None, None, None, None, 0.5, 0.2, 0.0, 1.0, None, None, None) == fem.FEM_ERR_ARG
    assert L.fem_mma_step(None, None, 0.0, None, None, 0.0, 1.0, 0, None, None, None, None, None, None,
                          None) == fem.FEM_ERR_ARG


def test_binding_struct_layouts_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    that a C compiler gives the same struct from include/fem.h."""
    import shutil
    import subprocess
    from paper_2212_00964_gb300 import fem
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    structs = [fem.fem_material, fem.fem_options, fem.fem_stats, fem.fem_bc, fem.fem_instance, fem.fem_j2_material]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "fem.h"', "int main(void) {"]
    for S in structs:
        n = S.__name__
        lines.append(f'printf("{n} size %zu\\n", sizeof({n}));')
        for f in S._fields_:
            lines.append(f'printf("{n} {f[0]} %zu\\n", offsetof({n}, {f[0]}));')
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for S in structs:
        n = S.__name__
        assert got[(n, "size")] == ctypes.sizeof(S), n
        for f in S._fields_:
            assert got[(n, f[0])] == getattr(S, f[0]).offset, (n, f[0])
