"""Build libens.so (the CUDA library behind include/ens.h) in-tree with nvcc.

sm_103a only: ``-gencode arch=compute_103a,code=sm_103a``.  The translation
units compile in parallel and link into ``paper_2506_23712_gb300/libens.so``
(static CUDA runtime, so the library does not depend on the toolkit's
libcudart at run time).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libens.so")
SOURCES = ["ens_kernels.cu", "ens_api.cu", "ens_noalloc.cu", "ens_surrogate.cu", "ens_theory.cu"]
# the persistent stage kernel reads, within one launch, data other CTAs wrote:
# its global loads are cached in L2 only
PERSIST = "ens_persist.cu"
PERSIST_FLAGS = ["-Xptxas", "-dlcm=cg"]
# the FFT passes of each grid size compile in their own translation unit
SIZED = "ens_sized.cu"
SIZES = [16, 32, 64, 128, 256, 384, 512]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-diag-suppress", "177",
         "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libens")


def _inputs():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(ROOT, "include", "ens.h"))
    deps.append(os.path.abspath(__file__))
    return deps


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(job):
        src, defs, obj = job
        obj = os.path.join(BUILD, obj)
        cmd = [cc] + ARCH + FLAGS + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr))
        if verbose and r.stderr.strip():
            sys.stderr.write(r.stderr)
        return obj

    jobs = [(SIZED, ["-DENS_N=%d" % n], "ens_sized_%d.o" % n) for n in reversed(SIZES)]
    jobs += [(PERSIST, PERSIST_FLAGS, PERSIST.replace(".cu", ".o"))]
    jobs += [(src, [], src.replace(".cu", ".o")) for src in SOURCES]
    with ThreadPoolExecutor(max_workers=min(len(jobs), max(2, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(compile_one, jobs))
    tmp = LIB + ".tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
