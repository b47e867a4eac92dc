"""Builds the sm_103a shared library ``liblbmtau1.so`` in-tree with nvcc.

Each translation unit is compiled in parallel for exactly one target,
``-gencode arch=compute_103a,code=sm_103a``, then linked with the shared CUDA
runtime (so the process shares one runtime, and its current device, with
PyTorch).
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "liblbmtau1.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["lbm_step_f32.cu", "lbm_step_f16.cu", "lbm_step_bf16.cu",
           "lbm_step.cu", "lbm_api.cu", "lbm_noalloc.cu", "lbm_batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    path = os.path.join(home, "bin", "nvcc")
    return path if os.path.exists(path) else "nvcc"


def _cuda_lib() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    for d in ("lib64", os.path.join("targets", "sbsa-linux", "lib"),
              os.path.join("targets", "x86_64-linux", "lib")):
        p = os.path.join(home, d)
        if os.path.exists(os.path.join(p, "libcudart.so")):
            return p
    return os.path.join(home, "lib64")


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC)
              if f.endswith((".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "lbmtau1.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", INCLUDE]

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.run(cmd, check=True, capture_output=not verbose)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp%d" % os.getpid()
    libdir = _cuda_lib()
    subprocess.run([nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp]
                   + objs + ["-L", libdir, "-Xlinker", "-rpath=" + libdir],
                   check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
