"""In-tree build of libkfbi.so (the CUDA library behind include/kfbi.h) for sm_103a.

Each translation unit is compiled by its own nvcc process in parallel, then linked with
`nvcc -shared`.  Run as `python -m paper_2404_15249_gb300.build` or through
`__graft_entry__.build()`.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libkfbi.so")
SOURCES = ["dst.cu", "dst_f32.cu", "dst_f64.cu", "setup2d.cu", "apply2d.cu", "gmres.cu", "capi.cu",
           "box_static.cu", "kfbi3d.cu", "dst3d.cu", "dst_tc.cu", "dst_tri.cu", "dst_ycol.cu", "probe.cu"]
ARCH = os.environ.get("KFBI_ARCH", "103a")


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         f"-gencode=arch=compute_{ARCH},code=sm_{ARCH}", "-diag-suppress", "177"]


def _compile(src: str) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared", f"-gencode=arch=compute_{ARCH},code=sm_{ARCH}", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
