"""Compile libwf (the CUDA kernels behind include/wf.h) for sm_103a, in tree.

Each .cu file under csrc/ is compiled by nvcc in parallel and the objects are
linked into ``_lib/libwf.so``.  ``-Xptxas -v`` resource usage (registers,
shared memory, spills) is kept in ``_lib/ptxas.log``.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libwf.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libwf")


def _stale(sources, target) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    deps = sources + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "wf.h"),
                                                               __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    if not force and not _stale(sources, LIB):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = [ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
              "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-Xptxas", "-v"]
    tag = f"{os.getpid()}"

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src) + f".{tag}.o")
        r = subprocess.run([nvcc, *common, "-c", src, "-o", obj], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max(1, min(len(sources), os.cpu_count() or 4))) as ex:
        results = list(ex.map(compile_one, sources))
    objs = [o for o, _ in results]
    with open(os.path.join(OUT_DIR, "ptxas.log"), "w") as f:
        for src, (_, log) in zip(sources, results):
            f.write(f"== {os.path.basename(src)}\n{log}\n")
    tmp = LIB + f".{tag}.tmp"
    r = subprocess.run([nvcc, ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
