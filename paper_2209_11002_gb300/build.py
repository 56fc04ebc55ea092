"""Builds libedaa.so (the C-ABI library) in-tree with nvcc for sm_103a.

Each .cu translation unit is compiled in its own nvcc process (in parallel),
then linked into paper_2209_11002_gb300/lib/libedaa.so with the CUDA runtime
linked statically, so the library loads on machines without a GPU driver
(compute calls then fail with EDAA_ERR_CUDA).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "lib")
OBJ_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libedaa.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (source, extra flags, object name); the pass bodies compile once per p
SOURCES = [("edaa_kernels.cu", [], "edaa_kernels"), ("edaa_capi.cu", [], "edaa_capi"),
           ("edaa_static.cu", [], "edaa_static"), ("edaa_unrolled.cu", [], "edaa_unrolled")] + [
    ("edaa_pass_p.cu", [f"-DEDAA_P={p}"], f"edaa_pass_p{p}") for p in range(1, 9)]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-rdc=true", "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the EDAA library needs the CUDA toolkit to build")
    return exe


def _compile(job, verbose: bool) -> str:
    src, flags, name = job
    obj = os.path.join(OBJ_DIR, name + ".o")
    cmd = [nvcc(), *ARCH, *COMMON, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        sys.stderr.write(r.stdout + r.stderr)
    return obj


def build_library(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(OBJ_DIR, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "edaa.h"))
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(d) for d in deps)
        if os.path.getmtime(LIB) >= newest:
            return LIB
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-rdc=true", "-shared", "-cudart", "static", "-Xcompiler", "-fPIC", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_library(verbose="-v" in sys.argv, force=True))
