"""Build liblightfuse.so (all CUDA sources, sm_103a) into this package directory."""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "liblightfuse.so")
# the same sources with the device bounds checks compiled in (LF_CHECKED)
CHECKED_LIB = os.path.join(HERE, "liblightfuse_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in deps())


def build(force: bool = False, verbose: bool = False, extra=(), out: str = LIB) -> str:
    if not force and not stale(out):
        return out
    nvcc = os.environ.get("NVCC", "nvcc")
    tmp = out + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
           "-Xlinker", "-rpath,/usr/local/cuda/lib64", f"-I{INCLUDE}", *extra, *sources(), "-o", tmp]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def build_checked(force: bool = False, verbose: bool = False) -> str:
    """The library with its device bounds checks (LF_CHECKED): a failed check
    reports LF_ERR_BOUNDS and skips the access instead of touching memory."""
    return build(force=force, verbose=verbose, extra=("-DLF_CHECKED=1",), out=CHECKED_LIB)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
    if "--checked" in sys.argv:
        print(build_checked(force="--force" in sys.argv, verbose=True))
