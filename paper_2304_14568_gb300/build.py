"""Build librpt.so in-tree with nvcc for sm_103a (no cmake, no torch extension).

The translation units compile in parallel; the shared library links the
CUDA runtime statically.  Run `python -m paper_2304_14568_gb300.build`.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librpt.so")
SOURCES = ["rowpass.cu", "rowstream.cu", "solver.cu", "api.cu", "noalloc.cu", "mlp.cu", "chol.cu", "dosecon.cu"]
HEADERS = ["common.cuh", "rowcommon.cuh", "gemm.cuh", "gemm_bf16.cuh", "gemm_tf32.cuh", "plan.h", "layout.h", "chunk.h", "batch.h", os.path.join("..", "..", "include", "rpt.h")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths if os.path.exists(p))


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"command failed ({r.returncode}): {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.normpath(os.path.join(CSRC, h)) for h in HEADERS]
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest(deps):
        return LIB
    objs = [os.path.join(BUILD, os.path.splitext(s)[0] + ".o") for s in SOURCES]

    def compile_one(i):
        return _run([NVCC, *FLAGS, "-c", srcs[i], "-o", objs[i]])

    with ThreadPoolExecutor(len(srcs)) as ex:
        logs = list(ex.map(compile_one, range(len(srcs))))
    tmp = LIB + ".tmp"
    logs.append(_run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs]))
    os.replace(tmp, LIB)
    if verbose:
        sys.stdout.write("".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
