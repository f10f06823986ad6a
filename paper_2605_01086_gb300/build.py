"""Builds libfptc.so in-tree for sm_103a (nvcc for the kernels, g++ for the host code)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build", "fptc")
LIB = os.path.join(PKG, "libfptc.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["index.cu", "decode.cu", "decode_fixed.cu", "decode_warp.cu", "decode_shape.cu", "decode_tc.cu", "decode_tcs.cu", "backward.cu",
              "backward_warp.cu", "decode_paper.cu",
              "noalloc.cu", "encode.cu", "wait_check.cu"]
CPP_SOURCES = ["plan.cpp", "codec_host.cpp"]


def _nvcc():
    p = os.path.join(CUDA_HOME, "bin", "nvcc")
    return p if os.path.exists(p) else shutil.which("nvcc")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + \
            [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)] + [os.path.abspath(__file__)]
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str) -> str:
    obj = os.path.join(BUILD, src + ".o")
    inc = ["-I", INCLUDE, "-I", CSRC]
    if src.endswith(".cu"):
        cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-Xptxas", "-warn-spills", *inc, "-c", os.path.join(CSRC, src), "-o", obj]
    else:
        cmd = ["g++", "-O2", "-fPIC", "-std=c++17", "-ffp-contract=off", "-Wall", *inc,
               "-I", os.path.join(CUDA_HOME, "include"), "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compiling {src} failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False) -> str:
    """Compile every translation unit in parallel and link libfptc.so next to the package."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    if _nvcc() is None:
        raise RuntimeError("nvcc not found: set CUDA_HOME")
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(CU_SOURCES) + len(CPP_SOURCES)) as ex:
        objs = list(ex.map(_compile, CU_SOURCES + CPP_SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath", "-Xlinker", os.path.join(CUDA_HOME, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"linking libfptc.so failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
