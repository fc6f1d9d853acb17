"""Build liblbfe.so in-tree for sm_103a (nvcc; the translation units compile in parallel).

Usage: ``python -m paper_2008_01473_gb300.build`` or ``build()`` from Python.
The library lands in ``paper_2008_01473_gb300/_build/liblbfe.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblbfe.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"] + ARCH
CUDA_UNITS = ["step_f32.cu", "step_persist.cu", "step_f64.cu", "step_f64s.cu", "step_f32s.cu", "step_rows.cu",
              "step_f32_pair0.cu", "step_f32_pair1.cu", "step_f32_pair2.cu", "step_f32_pair3.cu",
              "step_f32_pair0s.cu", "step_f32_pair1s.cu", "step_f32_pair2s.cu", "step_f32_pair3s.cu",
              "lbfe_api.cu", "lbfe_static.cu"]
HOST_UNITS = ["thermo.cpp"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build liblbfe")
    return cand


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(HERE, "..", "include", "lbfe.h")]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    """Compile every unit (in parallel) and link ``liblbfe.so``; returns its path."""
    if not force and not stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    flags = NVCC_FLAGS + (extra_flags or [])
    procs = []
    objs = []
    for u in CUDA_UNITS:
        obj = os.path.join(OUT_DIR, u.replace(".cu", ".o"))
        cmd = [nvcc] + flags + ["-c", os.path.join(CSRC, u), "-o", obj]
        procs.append((u, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    for u in HOST_UNITS:
        obj = os.path.join(OUT_DIR, u.replace(".cpp", ".o"))
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-c", os.path.join(CSRC, u), "-o", obj]
        procs.append((u, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for u, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(u)
    if failed:
        raise RuntimeError(f"liblbfe build failed in {failed}")
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
    print(LIB)
