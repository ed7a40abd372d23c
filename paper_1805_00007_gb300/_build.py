"""Compile the CUDA library in-tree for sm_103a (nvcc, translation units in parallel, no cmake)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbch.so")
SOURCES = [os.path.join(CSRC, f) for f in ("lbch_api.cu", "lbch_sweep_f32.cu", "lbch_sweep_f64.cu",
                                          "lbch_sweep_f16s.cu", "lbch_sweep_f32_m3.cu", "lbch_sweep_f64_m3.cu",
                                          "lbch_sweep_f16s_m3.cu", "lbch_noalloc.cu", "lbch_pair.cu",
                                          "lbch_probe.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + [
    os.path.join(ROOT, "include", "lbch.h")]

COMPILE_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
                 "-Xcompiler", "-fPIC"]
LINK_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-shared"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile each translation unit to an object in parallel, then link the shared library."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in DEPS if os.path.exists(p))
        if os.path.getmtime(LIB) >= newest:
            return LIB
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + f".{os.getpid()}.o")
        cmd = [nvcc(), *COMPILE_FLAGS, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        objs.append(obj)
        procs.append((cmd, subprocess.Popen(cmd)))
    failed = [cmd for cmd, p in procs if p.wait() != 0]
    if failed:
        raise subprocess.CalledProcessError(1, failed[0])
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([nvcc(), *LINK_FLAGS, *objs, "-o", tmp], check=True)
    for obj in objs:
        os.remove(obj)
    os.replace(tmp, LIB)
    return LIB
