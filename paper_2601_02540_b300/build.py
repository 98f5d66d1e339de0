"""Build libsgn.so (the CUDA library behind include/sgn.h) in-tree for sm_103a,
and libsgn_checked.so, the same sources with -DSGN_CHECKED (poisoned shared
-memory tiles and index bounds checks, for tests).

    python -m paper_2601_02540_b300.build [--force] [-v]

nvcc cross-compiles without a GPU.  The libraries land next to this file so
that they travel with the source tree.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libsgn.so")
LIB_CHECKED = os.path.join(HERE, "libsgn_checked.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["sgn_api.cu", "sgn_noalloc.cu", "sgn_batch.cu", "sgn_rate.cu"]


def _sources() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return files


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _sources())


def _compile(lib: str, extra: list[str], verbose: bool) -> None:
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-I", INCLUDE, "-I", CSRC, *extra,
           "-Xcompiler", "-fPIC,-fvisibility=hidden", "-shared", "-o", lib + ".tmp",
           *[os.path.join(CSRC, s) for s in SOURCES], "-lcudart"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(lib + ".tmp", lib)


def build(force: bool = False, verbose: bool = False, checked: bool = True) -> str:
    if force or not up_to_date(LIB):
        _compile(LIB, [], verbose)
    if checked and (force or not up_to_date(LIB_CHECKED)):
        _compile(LIB_CHECKED, ["-DSGN_CHECKED"], False)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
