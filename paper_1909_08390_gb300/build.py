"""Build libfdlb.so in-tree for sm_103a (GB300).

The kernels (csrc/fdlb_kernels.cu) go through nvcc with a single
``-gencode arch=compute_103a,code=sm_103a``; the host API (csrc/fdlb_api.cpp)
through g++; both compile in parallel and are linked by nvcc against the shared CUDA
runtime (the one PyTorch loads), so device selection and streams are shared.  Objects go to ``_build/`` next to this file.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfdlb.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

SOURCES = ["fdlb_kernels.cu", "fdlb_mixed.cu", "fdlb_api.cpp", "fdlb_noalloc.cu", "fdlb_adjoint.cu",
           "fdlb_peak.cu"]
HEADERS = [os.path.join(CSRC, "fdlb_internal.h"), os.path.join(CSRC, "fdlb_ctx.h"),
           os.path.join(CSRC, "fdlb_device.cuh"),
           os.path.join(CSRC, "fdlb_mp9.cuh"), os.path.join(CSRC, "fdlb_tile.cuh"),
           os.path.join(INCLUDE, "fdlb.h")]


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.isdir(home):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    objs, procs = [], []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        if not force and not _stale(obj, [path] + HEADERS):
            continue
        if src.endswith(".cu"):
            cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-Xptxas", "-v" if verbose else "-O3", "-I", INCLUDE, "-I", CSRC, "-c", path,
                   "-o", obj]
        else:
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-I", INCLUDE, "-I", CSRC, "-I",
                   os.path.join(cuda, "include"), "-c", path, "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                                            text=True)))
    failed = False
    for cmd, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0 or verbose:
            sys.stderr.write(out)
        if pr.returncode != 0:
            sys.stderr.write("failed: " + " ".join(cmd) + "\n")
            failed = True
    if failed:
        raise RuntimeError("libfdlb build failed")
    if force or _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        # the shared CUDA runtime: one runtime instance per process, so the
        # library sees the device and streams PyTorch selected
        lib64 = os.path.join(cuda, "lib64")
        subprocess.run([nvcc, ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath",
                        "-Xlinker", lib64, "-o", tmp] + objs, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
