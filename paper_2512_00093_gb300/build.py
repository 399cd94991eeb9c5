"""Builds libranmar (the CUDA library behind include/ranmar.h) in-tree.

One translation unit, one -gencode (sm_103a), static cudart; the result is
paper_2512_00093_gb300/_build/libranmar.so.  No torch extension machinery:
the library exports a plain C ABI and the Python side loads it with ctypes.
"""
from __future__ import annotations

import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libranmar.so")
PROBE_LIB = os.path.join(BUILD, "libranmar_probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _sources() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)
             if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "ranmar.h"))
    return files


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: libranmar needs the CUDA toolkit to build")
    return exe


def _compile(src: str, out: str, deps: list[str], force: bool, verbose: bool):
    if not force and os.path.exists(out):
        t = os.path.getmtime(out)
        if all(os.path.getmtime(f) <= t for f in deps):
            return None
    os.makedirs(BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-shared", "-I", INCLUDE, "-o", tmp, src]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    return subprocess.Popen(cmd), tmp, out


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/ranmar.cu into _build/libranmar.so and csrc/probe.cu into
    _build/libranmar_probe.so (in parallel) if they are stale."""
    jobs = [_compile(os.path.join(CSRC, "ranmar.cu"), LIB,
                     [f for f in _sources() if not f.endswith("probe.cu")], force, verbose),
            _compile(os.path.join(CSRC, "probe.cu"), PROBE_LIB,
                     [os.path.join(CSRC, "probe.cu")], force, verbose)]
    for job in jobs:
        if job is None:
            continue
        proc, tmp, out = job
        if proc.wait() != 0:
            raise RuntimeError(f"nvcc failed building {out}")
        os.replace(tmp, out)
    return LIB


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
