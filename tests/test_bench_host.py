"""Host-side logic of bench.py (no GPU): the workload name shared by both
arms, and the guard that reports the ncu DRAM traffic only for the apply
kernel and the kernel sources the capture was taken on."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_workload_name_counts_dofs():
    b = load_bench()
    assert "(823875 DOF)" in b.workload_name(64)
    assert b.workload_name(8).startswith("Neo-Hookean 8^3")


def test_traffic_only_for_the_captured_kernel_and_sources():
    b = load_bench()
    b.APPLY_TRAFFIC_SHA256 = b.sources_hash()  # the capture describes these sources
    for k in range(1, 11):
        t = b.apply_traffic(k)
        assert (t is None) == (k not in b.APPLY_TRAFFIC_BYTES)
    k = next(iter(b.APPLY_TRAFFIC_BYTES))
    assert b.apply_traffic(k) == b.APPLY_TRAFFIC_BYTES[k]
    b.APPLY_TRAFFIC_SHA256 = "0" * 64  # sources changed since the capture
    assert b.apply_traffic(k) is None


def test_every_apply_kernel_has_a_flop_count_and_name():
    b = load_bench()
    assert set(b.APPLY_FLOPS_PER_CELL) == set(range(1, 13))
    assert all(0 < v <= b.NH_APPLY_FLOPS_PER_CELL for v in b.APPLY_FLOPS_PER_CELL.values())


def test_allocation_free_solve_tests_are_collected_last():
    """The fem_solve_static tests run after every other GPU test, so a stop
    on the first failure (-x) has already run all the others."""
    import subprocess
    import sys
    out = subprocess.run([sys.executable, "-m", "pytest", "--collect-only", "-q", "-m", "gpu", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests")], capture_output=True, text=True, cwd=ROOT).stdout
    ids = [l for l in out.splitlines() if "::" in l]
    last = [("test_zz_no_alloc.py" in l) for l in ids]
    assert any(last) and not all(last)
    first = last.index(True)
    assert all(last[first:]), "a GPU test is collected after the allocation-free solve tests"
