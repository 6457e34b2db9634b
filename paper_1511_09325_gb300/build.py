"""Compile the CUDA library ``libsnn_gb300.so`` in-tree for sm_103a.

Translation units are compiled in parallel (nvcc for the .cu files, g++ for
the host tables) and linked with nvcc.  ``-ffp-contract=off`` / ``-fmad=false``
keep every floating-point operation exactly as written, which the
bit-exactness of the fixed-point/FP32 mode relies on.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libsnn_gb300.so")
OBJDIR = os.path.join(PKG, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler",
              "-fPIC,-ffp-contract=off", "-I", INCLUDE, "-I", CSRC] + ARCH
GXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I", INCLUDE,
             "-I", CSRC]

CU_SOURCES = ["snn_build.cu", "snn_step.cu", "snn_api.cu", "snn_noalloc.cu", "snn_grad.cu"]
CXX_SOURCES = ["snn_tables.cpp"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _cuda_include():
    nv = _nvcc()
    base = os.path.dirname(os.path.dirname(nv)) if os.path.isabs(nv) else "/usr/local/cuda"
    return os.path.join(base, "include")


def _sources():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(INCLUDE, "snn.h"))
    deps.append(os.path.abspath(__file__))
    return deps


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _sources())


def build(force=False, verbose=False, extra_nvcc=()):
    """Build the shared library; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for src in CU_SOURCES:
        obj = os.path.join(OBJDIR, src + ".o")
        jobs.append([nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + NVCC_FLAGS + list(extra_nvcc))
    for src in CXX_SOURCES:
        obj = os.path.join(OBJDIR, src + ".o")
        jobs.append(["g++", "-c", os.path.join(CSRC, src), "-o", obj, "-I", _cuda_include()] + GXX_FLAGS)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        p = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, p

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(run, jobs))
    for cmd, p in results:
        if verbose and p.stderr:
            print(p.stderr, file=sys.stderr)
        if p.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), p.stdout, p.stderr))
    objs = [os.path.join(OBJDIR, s + ".o") for s in CU_SOURCES + CXX_SOURCES]
    tmp = LIB + ".tmp%d" % os.getpid()
    link = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    p = subprocess.run(link, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("link failed: %s\n%s%s" % (" ".join(link), p.stdout, p.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
