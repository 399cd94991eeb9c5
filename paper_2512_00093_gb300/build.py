"""Builds libranmar (the CUDA library behind include/ranmar.h) in-tree.

Two translation units compiled in parallel -- csrc/ranmar.cu (the kernels
and their entry points, one -gencode: sm_103a) and csrc/serve.cpp (the
serving scheduler, host code) -- linked with static cudart into
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
             if f.endswith((".cu", ".cuh", ".h")) and f != "probe.cu"]
    files.append(os.path.join(INCLUDE, "ranmar.h"))
    return files


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: libranmar needs the CUDA toolkit to build")
    return exe


def _stale(out: str, deps: list[str], force: bool) -> bool:
    if force or not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(f) > t for f in deps)


def _start(srcs: list[str], out: str, shared: bool, verbose: bool):
    os.makedirs(BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-shared" if shared else "-c", "-I", INCLUDE, "-o", tmp, *srcs]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    return subprocess.Popen(cmd), tmp, out


def _finish(jobs) -> None:
    failed = []
    for proc, tmp, out in jobs:
        if proc.wait() != 0:
            failed.append(out)
        else:
            os.replace(tmp, out)
    if failed:
        raise RuntimeError(f"nvcc failed building {', '.join(failed)}")


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/ranmar.cu and csrc/serve.cpp (in parallel with each other
    and with csrc/probe.cu -> _build/libranmar_probe.so) and link the first
    two into _build/libranmar.so, each step only if stale."""
    header = os.path.join(INCLUDE, "ranmar.h")
    kern_o = os.path.join(BUILD, "ranmar.o")
    serve_o = os.path.join(BUILD, "serve.o")
    serve_src = os.path.join(CSRC, "serve.cpp")
    probe_src = os.path.join(CSRC, "probe.cu")
    jobs = []
    if _stale(kern_o, [f for f in _sources() if not f.endswith(".cpp")], force):
        jobs.append(_start([os.path.join(CSRC, "ranmar.cu")], kern_o, False, verbose))
    if _stale(serve_o, [serve_src, header], force):
        jobs.append(_start([serve_src], serve_o, False, verbose))
    if _stale(PROBE_LIB, [probe_src], force):
        jobs.append(_start([probe_src], PROBE_LIB, True, verbose))
    _finish(jobs)
    if _stale(LIB, [kern_o, serve_o], force):
        _finish([_start([kern_o, serve_o], LIB, True, False)])
    return LIB


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
