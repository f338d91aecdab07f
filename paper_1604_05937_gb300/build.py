"""Builds the extmesh CUDA library (libextmesh.so) in-tree for sm_103a.

Each .cu translation unit is compiled in parallel with nvcc, then linked into
one shared library against the shared CUDA runtime (so it shares the runtime
state of the process, e.g. PyTorch's current device).  No CMake, no cached
system-wide install: the library sits next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libextmesh.so")
# the checked build: ext_api.cu with EXT_CHECKED (every stencil index range-
# checked on the device before a launch), the other units shared
LIB_CHECKED = os.path.join(HERE, "libextmesh_checked.so")
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "extmesh.h")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-Xcompiler", "-Wall"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")) + [HEADER])


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(LIB_CHECKED):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_CHECKED))
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compiles and links libextmesh.so; returns its path."""
    if not force and not extra and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    extra = list(extra or [])

    def compile_one(job) -> str:
        src, checked = job
        obj = os.path.join(BUILD, os.path.basename(src) + (".checked.o" if checked else ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra, *(["-DEXT_CHECKED"] if checked else []), "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        return obj

    api = os.path.join(CSRC, "ext_api.cu")
    jobs = [(src, False) for src in srcs] + [(api, True)]
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        objs = list(ex.map(compile_one, jobs))
    plain, checked = objs[:-1], [o for o in objs[:-1] if not o.endswith("ext_api.cu.o")] + [objs[-1]]
    for lib, parts in ((LIB, plain), (LIB_CHECKED, checked)):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *parts,
               "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
