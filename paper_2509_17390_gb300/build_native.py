"""Build libfgl.so in-tree (nvcc for sm_103a, g++ for host-only sources).

Translation units compile in parallel; the library links the CUDA runtime
statically, so it only needs the driver at run time.  `build(checked=True)`
builds the checked library instead (libfgl_checked.so, -DFGL_CHECKED: the
traversal kernels compare every node and triangle index with the scene's
record counts before reading and report FGL_ERR_DEVICE instead of reading
out of range), the debugging stand-in for a memory checker.
"""

from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libfgl.so")
BUILD_CHECKED = os.path.join(PKG, "_build_checked")
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libfgl_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-I" + INCLUDE, "-I" + CSRC]
GXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math", "-pthread",
             "-I" + INCLUDE, "-I" + CSRC]

CU_SOURCES = ["kernels.cu", "api.cu", "static_batch.cu", "server.cu", "density.cu", "sort.cu", "lbvh.cu",
              "mesh.cu", "effects.cu"]
CPP_SOURCES = ["bvh_build.cpp"]
HEADERS = ["fgl_internal.h", "kernels.h", "trace.cuh", "ptx_ops.cuh", "sort.h", "nvtx_range.h"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile every translation unit that changed and link libfgl.so (or,
    with checked=True, libfgl_checked.so)."""
    build_dir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    os.makedirs(build_dir, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "fgl.h")]
    jobs, objs = [], []
    nvcc = _nvcc()
    for src in CU_SOURCES + CPP_SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(build_dir, src + ".o")
        objs.append(obj)
        if force or _stale(obj, [path] + hdrs):
            if src.endswith(".cu"):
                cmd = [nvcc] + NVCC_FLAGS + (["-DFGL_CHECKED=1"] if checked else []) + ["-c", path, "-o", obj]
            else:
                cmd = ["g++"] + GXX_FLAGS + ["-c", path, "-o", obj]
            jobs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in jobs:
        out, _ = p.communicate()
        if p.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
            raise RuntimeError("compilation failed: " + " ".join(cmd))
        if verbose and out:
            sys.stderr.write(out.decode(errors="replace"))
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-Xcompiler", "-pthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
