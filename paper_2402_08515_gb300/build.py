"""In-tree build of libkes.so for sm_103a (GB300).

Each translation unit is compiled by its own nvcc process (in parallel) and
linked into ``paper_2402_08515_gb300/libkes.so`` with the CUDA runtime linked
statically, so the library loads on a machine without a GPU (its CUDA calls
then fail with KES_ERR_CUDA). Run ``python paper_2402_08515_gb300/build.py`` (the package itself needs the library).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libkes.so")
SOURCES = [
    "csrc/host_math.cpp",
    "csrc/sell.cpp",
    "csrc/kernels_step.cu",
    "csrc/kernels_blas.cu",
    "csrc/kernels_block.cu",
    "csrc/kes_api.cu",
    "csrc/solver.cu",
    "csrc/noalloc.cu",
]
HEADERS = ["csrc/kes_internal.h", "csrc/kes_ctx.h", os.path.join("..", "include", "kes.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkes.so")


def _flags():
    return ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O3,-fopenmp",
            "-I", os.path.join(ROOT, "include"), "-I", os.path.join(HERE, "csrc")]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    for rel in SOURCES + HEADERS + [os.path.relpath(__file__, HERE)]:
        if os.path.getmtime(os.path.join(HERE, rel)) > t:
            return True
    return False


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libkes.so if a source is newer than it (or ``force``); returns its path."""
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD_DIR, exist_ok=True)

    def compile_one(rel):
        src = os.path.join(HERE, rel)
        obj = os.path.join(BUILD_DIR, os.path.basename(rel) + ".o")
        cmd = [nvcc, *_flags(), "-c", src, "-o", obj]
        if verbose and rel.endswith(".cu"):
            cmd += ["-Xptxas", "-v"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed on {rel}:\n{p.stdout}\n{p.stderr}")
        return obj, p.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for (_, log), rel in zip(results, SOURCES):
            if log.strip():
                print(f"--- {rel}\n{log}", file=sys.stderr)
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fopenmp", "-o", tmp, *[o for o, _ in results], "-lgomp"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stdout}\n{p.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
