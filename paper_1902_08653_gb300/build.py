"""Builds the CUDA library (libcdmimo.so) in-tree for sm_103a with nvcc.

Each csrc/*.cu file is one translation unit (kernels are header templates instantiated where they
are launched); the units compile in parallel with a single -gencode and are linked into one
shared library, so the build stays around a minute.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "_build", "libcdmimo.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcdmimo.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date() -> bool:
    if not os.path.exists(OUT):
        return False
    t = os.path.getmtime(OUT)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _run(cmd):
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
    return res.stdout + res.stderr


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and up_to_date():
        return OUT
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    tag = f"{os.getpid()}"
    common = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
              *extra]
    if verbose:
        common.insert(1, "-Xptxas=-v")
    objs, cmds = [], []
    for src in sources():
        obj = os.path.join(os.path.dirname(OUT), os.path.basename(src)[:-3] + f".{tag}.o")
        objs.append(obj)
        cmds.append([*common, "-c", "-o", obj, src])
    try:
        with cf.ThreadPoolExecutor(len(cmds)) as ex:
            logs = list(ex.map(_run, cmds))
        tmp = OUT + f".{tag}.tmp"
        _run([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, OUT)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    if verbose:
        print("".join(logs))
    return OUT


if __name__ == "__main__":
    print(build(force=True, verbose=True))
