"""Build the CUDA library ``libdmr.so`` in-tree for sm_103a (GB300).

Two translation units compiled in parallel with nvcc, linked into one
shared library against the shared CUDA runtime (the one PyTorch loads), so
device pointers and streams are interchangeable with torch's.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdmr.so")
SOURCES = ["dmr_api.cu", "dmr_kernels.cu", "dmr_noalloc.cu", "dmr_raster_f32.cu", "dmr_raster_bf16.cu",
           "dmr_raster_f16.cu", "dmr_hv.cpp", "dmr_mlp.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "dmr.h"))
    return files


def build_library(force: bool = False, verbose: bool = False, ptxas_v: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in _deps())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if ptxas_v:
        common += ["-Xptxas", "-v"]
    if os.environ.get("DMR_RASTER_THREADS_PER_SM"):
        common += ["-DDMR_RASTER_THREADS_PER_SM=%d" % int(os.environ["DMR_RASTER_THREADS_PER_SM"])]
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        objs.append(obj)
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for cmd, pr in procs:
        out, _ = pr.communicate()
        text = out.decode(errors="replace")
        if pr.returncode != 0:
            errors.append(" ".join(cmd) + "\n" + text)
        elif verbose or ptxas_v:
            print(text, file=sys.stderr)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = LIB + ".%d.tmp" % os.getpid()
    link = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
    subprocess.check_call(link)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build_library(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv)
    print(LIB)
