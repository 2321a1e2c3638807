"""Builds of the host harnesses (tests/*_host.cpp) that compile the CUDA
library's host/device arithmetic and control code for the CPU.  With
FEMGB_HOST_SANITIZE=1 they are built with AddressSanitizer and
UndefinedBehaviorSanitizer into separate files (the process must then run
with the ASan runtime preloaded; tests/test_host_sanitizers.py does that)."""
import ctypes
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT = os.path.join(ROOT, "paper_2212_00964_gb300", "_lib")
CSRC = os.path.join(ROOT, "paper_2212_00964_gb300", "csrc")
SANITIZE = os.environ.get("FEMGB_HOST_SANITIZE") == "1"


def build(name, extra_deps=(), extra_flags=()):
    """Compile tests/<name>.cpp into _lib/<name>.so (or <name>_san.so) if
    stale; returns the loaded library."""
    src = os.path.join(HERE, name + ".cpp")
    so = os.path.join(OUT, name + ("_san.so" if SANITIZE else ".so"))
    deps = [src] + [os.path.join(CSRC, d) for d in os.listdir(CSRC)] + [os.path.join(HERE, "cpu_pcg.h")]
    deps += list(extra_deps)
    os.makedirs(OUT, exist_ok=True)
    if not os.path.exists(so) or os.path.getmtime(so) < max(os.path.getmtime(f) for f in deps if os.path.exists(f)):
        tmp = so + ".tmp%d" % os.getpid()
        flags = ["-std=c++17", "-fPIC", "-shared", "-Wall"] + list(extra_flags)
        if SANITIZE:
            flags += ["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                      "-fno-sanitize-recover=all"]
        else:
            flags += ["-O2"]
        subprocess.check_call(["g++"] + flags + [src, "-o", tmp])
        os.replace(tmp, so)
    return ctypes.CDLL(so)
