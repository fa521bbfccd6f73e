"""Builds libsdgr.so (all CUDA kernels + the C ABI) for sm_103a, in-tree.

    python -m paper_2506_21633_b300.build            # build if stale
    python -m paper_2506_21633_b300.build --force    # rebuild
    python -m paper_2506_21633_b300.build --checked  # libsdgr_checked.so: index checks on

The checked library (-DSDGR_CHECKED) verifies the indices the binning and
raster stages produce against their buffers and reports a bad one through
the status word (SDGR_ERR_BOUNDS); SDGR_CHECKED=1 in the environment makes
the Python binding load it instead of libsdgr.so.

nvcc cross-compiles without a GPU.  Extra nvcc flags can be appended through
the SDGR_NVCC_FLAGS environment variable (e.g. "-Xptxas -v").
"""
from __future__ import annotations

import glob
import os
import shlex
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libsdgr.so")
LIB_CHECKED = os.path.join(PKG, "libsdgr_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc(), "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
           "-I", INCLUDE, "-o", tmp, *sources()]
    if checked:
        cmd.append("-DSDGR_CHECKED")
    cmd += shlex.split(os.environ.get("SDGR_NVCC_FLAGS", ""))
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
