"""Build libgenesys.so (runtime + sm_103a kernels) in-tree with nvcc.

    python -m paper_1705_06965_b300.build                  # libgenesys.so
    python -m paper_1705_06965_b300.build --device-checks  # libgenesys_checked.so

The checked library compiles the device-side index checks
(GENESYS_DEVICE_CHECKS: a failed check is counted in a status word instead of
faulting); the binding loads it when GENESYS_LIBRARY=checked.
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libgenesys.so")
LIB_CHECKED = os.path.join(PKG, "libgenesys_checked.so")

SOURCES = ["runtime.cpp", "workloads.cu", "wordcount.cu", "serve.cu", "kv.cu", "echo.cu"]
HEADERS = [os.path.join(INCLUDE, h) for h in ("genesys.h", "genesys_layout.h", "genesys_device.cuh")] + [
    os.path.join(CSRC, "internal.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for p in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if p and (os.path.isabs(p) and os.path.exists(p) or not os.path.isabs(p)):
            return p
    return "nvcc"


def command(out: str = LIB, extra: list[str] | None = None) -> list[str]:
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    return [nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
            "-shared", "-cudart", "shared", f"-I{INCLUDE}", f"-I{CSRC}", "-o", out, *srcs, "-lpthread",
            *(extra or [])]


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + HEADERS
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, device_checks: bool = False) -> str:
    lib = LIB_CHECKED if device_checks else LIB
    if force or stale(lib):
        extra = ["-Xptxas", "-v"] if verbose else []
        if device_checks:
            extra.append("-DGENESYS_DEVICE_CHECKS")
        r = subprocess.run(command(lib, extra), capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
        if verbose:
            print(r.stdout + r.stderr)
        elif "warning" in r.stderr:
            print(r.stderr, file=sys.stderr)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                device_checks="--device-checks" in sys.argv))
