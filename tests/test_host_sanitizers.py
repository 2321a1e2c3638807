"""The host builds of the CUDA library's arithmetic and control code
(tests/*_host.cpp) and the oracle's C code, run under AddressSanitizer and
UndefinedBehaviorSanitizer: every index the kernels' per-node, per-cell and
per-variable code computes, and every host-side control path the tests
drive, stays inside its buffers and free of undefined behaviour.  Each
sanitized run is a child process with the ASan runtime preloaded."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS_TESTS = ["test_poisson_core.py", "test_j2_core.py", "test_topopt_core.py", "test_dpcg_control.py",
                 "test_j2_step_host.py", "test_poisson_solve_host.py", "test_host_properties.py"]
ORACLE_TESTS = ["test_oracle_element.py", "test_oracle_global.py", "test_oracle_mesh.py", "test_oracle_solve.py",
                "test_oracle_poisson.py", "test_oracle_plasticity.py", "test_oracle_topopt.py", "test_golden.py"]


def _asan_runtime():
    cc = shutil.which("gcc")
    if cc is None:
        return None
    path = subprocess.run([cc, "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


def _run(files):
    rt = _asan_runtime()
    if rt is None:
        pytest.skip("no AddressSanitizer runtime")
    env = dict(os.environ, LD_PRELOAD=rt, ASAN_OPTIONS="detect_leaks=0", FEMGB_HOST_SANITIZE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider"] +
                       [os.path.join(ROOT, "tests", f) for f in files], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]


def test_kernel_host_builds_under_sanitizers():
    _run(HARNESS_TESTS)


@pytest.mark.slow
def test_oracle_under_sanitizers():
    _run(ORACLE_TESTS)
