"""Builds libotoo.so in the package directory (host C++ with g++/OpenMP,
device code with nvcc for sm_103a), translation units compiled in parallel."""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libotoo.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
HOST_SRC = ["host/tree.cpp"]
CUDA_HDR = ["cuda/force_warp.cuh", "cuda/force_warp2.cuh", "cuda/pair.cuh"]
CUDA_SRC = ["cuda/force.cu", "cuda/mlp.cu", "cuda/direct.cu", "cuda/walk.cu", "cuda/tree_build.cu", "cuda/sph.cu",
            "cuda/peak.cu"]


def _nvcc():
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _cuda_home():
    nv = _nvcc()
    if os.path.isabs(nv):
        return os.path.dirname(os.path.dirname(os.path.realpath(nv)))
    return os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n%s\n%s" % (" ".join(cmd), r.stdout))
    return r.stdout


def sources():
    return [os.path.join(CSRC, s) for s in HOST_SRC + CUDA_SRC + CUDA_HDR] + [os.path.join(CSRC, "common.h"),
                                                                   os.path.join(CSRC, "treegeom.h"), os.path.join(CSRC, "plan_chunks.h"),
                                                                   os.path.join(INCLUDE, "otoo.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force=False, verbose=False, ptxas_info=False):
    """Compile and link libotoo.so; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    objs = []
    for s in HOST_SRC:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        objs.append(o)
        jobs.append(["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-ffp-contract=off", "-I" + INCLUDE,
                     "-I" + os.path.join(_cuda_home(), "include"), "-c", os.path.join(CSRC, s), "-o", o])
    for s in CUDA_SRC:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        objs.append(o)
        cmd = [_nvcc()] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE,
                                  "-c", os.path.join(CSRC, s), "-o", o]
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        jobs.append(cmd)
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    tmp = LIB + ".tmp%d" % os.getpid()
    _run([_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-Xcompiler", "-fopenmp", "-lgomp"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    build(force=True, verbose=True, ptxas_info="-v" in sys.argv)
    print(LIB)
