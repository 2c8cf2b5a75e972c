"""Build the CUDA library in-tree: paper_1909_06935_gb300/_build/libmrq.so (sm_103a only)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC_DIR = os.path.join(HERE, "csrc")
SOURCES = [os.path.join(SRC_DIR, "mrq.cu"), os.path.join(SRC_DIR, "mrq_probe.cu"),
           os.path.join(SRC_DIR, "mrq_sci.cu"), os.path.join(SRC_DIR, "mrq_server.cpp")]
DEPS = SOURCES + [os.path.join(SRC_DIR, "mrq_device.cuh"), os.path.join(SRC_DIR, "mrq_cas.cuh"),
                  os.path.join(SRC_DIR, "mrq_walk.cuh"), os.path.join(SRC_DIR, "mrq_internal.h"),
                  os.path.join(os.path.dirname(HERE), "include", "mrq.h")]
LIB = os.path.join(HERE, "_build", "libmrq.so")
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    newest = max(os.path.getmtime(p) for p in DEPS)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc()] + NVCC_FLAGS + (["-Xptxas", "-v"] if verbose else []) + ["-Xcompiler", "-pthread", "-o", tmp] + SOURCES
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
