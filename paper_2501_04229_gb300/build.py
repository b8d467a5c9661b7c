"""Build libgadi.so in-tree with nvcc for sm_103a (GB300).

    python -m paper_2501_04229_gb300.build [--force] [-v]

The library is plain CUDA C++ behind the C ABI of include/gadi.h; it links
the CUDA runtime statically and has no PyTorch dependency. Translation
units are compiled in parallel, then linked.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libgadi.so")
OBJDIR = os.path.join(HERE, "_build")
SOURCES = ["gadi_api.cu", "gadi_noalloc.cu", "gadi_sweep.cu", "gadi_predict.cu", "gadi_sylvester.cu"]
HEADERS = ["gadi_solve.cuh", "gadi_ops.cuh", "gadi_device.cuh", "gadi_bits.cuh"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
# host code without floating-point contraction: set-up and stop-test arithmetic
# rounds each product and sum as written, on x86 and Arm alike
FLAGS = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler",
         "-fvisibility=hidden", "-Xcompiler", "-ffp-contract=off", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is needed to build libgadi.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + \
        [os.path.join(ROOT, "include", "gadi.h"), os.path.abspath(__file__)]
    return any(os.path.getmtime(f) > t for f in files)


def _run(cmd):
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
    return res.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    tag = f".{os.getpid()}"
    objs, cmds = [], []
    for src in SOURCES:
        obj = os.path.join(OBJDIR, os.path.splitext(src)[0] + tag + ".o")
        cmd = [nvcc(), *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        objs.append(obj)
        cmds.append(cmd)
    with cf.ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        logs = list(ex.map(_run, cmds))
    if verbose:
        for lg in logs:
            sys.stderr.write(lg)
    tmp = LIB + tag
    _run([nvcc(), ARCH, "-shared", "-cudart", "static", *objs, "-o", tmp])
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
