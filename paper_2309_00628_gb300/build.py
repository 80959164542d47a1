"""Build libswmm.so (CUDA, sm_103a) in-tree with nvcc.

Each translation unit compiles in parallel to an object file; the shared library is
named by a hash of the sources and flags, so a stale build is never loaded.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libswmm")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _tag() -> str:
    h = hashlib.sha1()
    for f in sources() + sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))) + [
            os.path.join(INCLUDE, "swmm.h")]:
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()[:12]


def lib_path() -> str:
    return os.path.join(OUT, f"libswmm_{_tag()}.so")


def build(force: bool = False, verbose: bool = False) -> str:
    so = lib_path()
    if os.path.exists(so) and not force:
        return so
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    tag = _tag()
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT, os.path.basename(src)[:-3] + f"_{tag}.o")
        cmd = [nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(sources())) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = so + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, so)
    # object files and libraries of older source versions are never loaded again
    for f in glob.glob(os.path.join(OUT, "*.o")) + glob.glob(os.path.join(OUT, "libswmm_*.so")):
        if f != so:
            try:
                os.remove(f)
            except OSError:
                pass
    return so


if __name__ == "__main__":
    print(build(verbose=True))
