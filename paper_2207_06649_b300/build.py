"""Build libpmbs.so in-tree with nvcc for sm_103a (B300), and its bounds-checked twin
libpmbs_checked.so (the same source compiled with -DPMBS_BOUNDS_CHECK=1: every shared
and global index of the rollout kernel checked, violations recorded in a status word read
by pmbs_check_status)."""
from __future__ import annotations

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libpmbs.so")
LIB_CHECKED = os.path.join(HERE, "libpmbs_checked.so")
SRC = os.path.join(HERE, "csrc", "pmbs_engine.cu")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-shared"]


def _sources():
    return [SRC] + glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + \
        [os.path.join(os.path.dirname(HERE), "include", "pmbs.h")]


def stale(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    if force or stale(checked):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [NVCC] + FLAGS + (["-DPMBS_BOUNDS_CHECK=1"] if checked else []) + \
            (["-Xptxas", "-v"] if verbose else []) + ["-o", tmp, SRC]
        subprocess.check_call(cmd)
        os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> None:
    """Both libraries (the two nvcc runs in parallel)."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(2) as ex:
        for f in [ex.submit(build, force, False, c) for c in (False, True)]:
            f.result()


if __name__ == "__main__":
    import sys
    build(force=True, verbose=True, checked="--checked" in sys.argv)
    print(LIB_CHECKED if "--checked" in sys.argv else LIB)
