"""Build step: compile the CUDA sources into the in-tree shared library
paper_1310_6736_b300/libks.so for sm_103a (B300) with nvcc.

    python -m paper_1310_6736_b300.build [--force] [--verbose-ptxas]
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libks.so")
INCLUDE = os.path.join(ROOT, "include")

OBJ_DIR = os.path.join(PKG, "_build")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17", "-fmad=false",
    "-Xcompiler", "-fPIC,-O2",
    "-I", INCLUDE, "-I", CSRC,
]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) \
        + [os.path.join(INCLUDE, "ks.h")]


def _obj(src):
    return os.path.join(OBJ_DIR, os.path.basename(src)[:-3] + ".o")


def _newer(deps, target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _stale():
    return _newer(sources() + _headers(), LIB)


def build(force=False, ptxas_verbose=False):
    """Compile libks.so if any source is newer than it; returns its path.
    Each translation unit is compiled to its own object (in parallel, only
    the ones whose source or a header changed), then the objects are
    linked into the shared library."""
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    os.makedirs(OBJ_DIR, exist_ok=True)
    hdrs = _headers()
    todo = [src for src in sources() if force or ptxas_verbose or _newer([src] + hdrs, _obj(src))]

    def compile_one(src):
        tmp = _obj(src) + f".tmp{os.getpid()}"
        cmd = [nvcc, *NVCC_FLAGS, "-c", "-o", tmp, src]
        if ptxas_verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, _obj(src))
        return src, r

    failed = []
    with ThreadPoolExecutor(max_workers=max(1, min(len(todo), os.cpu_count() or 4))) as pool:
        for src, r in pool.map(compile_one, todo):
            if r.returncode != 0:
                failed.append(src)
                sys.stderr.write(r.stdout + r.stderr)
            elif ptxas_verbose:
                sys.stderr.write(r.stderr)
    if failed:
        raise RuntimeError("nvcc failed building libks.so: " + ", ".join(map(os.path.basename, failed)))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp,
           *[_obj(src) for src in sources()], "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed linking libks.so")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, ptxas_verbose="--verbose-ptxas" in sys.argv)
    print(LIB)
