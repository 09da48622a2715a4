"""Compile the CUDA library in-tree for sm_103a (GB300).

    python -m paper_1902_02999_gb300.build

produces paper_1902_02999_gb300/_build/libmaclab.so from csrc/ (one nvcc
compile per translation unit, run side by side, then one link;
-gencode arch=compute_103a,code=sm_103a, -O3, -lineinfo).
"""
from __future__ import annotations

import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libmaclab.so")
SOURCES = [os.path.join(CSRC, "maclab.cu"), os.path.join(CSRC, "warmstart.cu")]
DEPENDS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")] + \
    [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(f) <= t for f in DEPENDS):
            return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    # one object per translation unit, compiled side by side, then linked
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(BUILD, os.path.splitext(os.path.basename(src))[0] + ".%d.o" % os.getpid())
        cmd = [nvcc(), "-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-c",
               "-I" + INCLUDE, "-o", obj, src]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        objs.append(obj)
        procs.append(subprocess.Popen(cmd))
    codes = [p.wait() for p in procs]
    try:
        if any(codes):
            raise subprocess.CalledProcessError(max(codes), "nvcc")
        subprocess.check_call([nvcc(), ARCH, "-shared", "-o", tmp] + objs)
    finally:
        for obj in objs:
            if os.path.exists(obj):
                os.remove(obj)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
