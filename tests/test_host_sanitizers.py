"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer: the CPU
oracle (oracle/fdlb_oracle.c) and the library's host API
(csrc/fdlb_api.cpp, with stand-ins for the kernel launchers) are compiled
with -fsanitize=address,undefined and driven through every entry point on
small, degenerate and rejected inputs (tests/host/*_sanitize.*).  A
sanitizer report aborts the driver; the test also fails on any report in its
output."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "host", "_build")
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer",
       "-g", "-O1"]


def _cuda_home():
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _run(exe):
    env = dict(os.environ, OMP_NUM_THREADS="2",
               ASAN_OPTIONS="detect_leaks=1:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=600)
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-4000:]
    assert "runtime error" not in out and "AddressSanitizer" not in out, out[-4000:]
    return out


def test_oracle_under_sanitizers():
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "oracle_sanitize")
    subprocess.run(["gcc", "-std=c11", "-ffp-contract=off", "-fopenmp"] + SAN +
                   [os.path.join(HERE, "host", "oracle_sanitize.c"),
                    os.path.join(ROOT, "oracle", "fdlb_oracle.c"), "-o", exe, "-lm"], check=True)
    assert "ok" in _run(exe)


def test_host_api_under_sanitizers():
    cuda = _cuda_home()
    lib64 = os.path.join(cuda, "lib64")
    if not os.path.exists(os.path.join(cuda, "include", "cuda_runtime.h")):
        pytest.skip("CUDA headers not found")
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "api_sanitize")
    csrc = os.path.join(ROOT, "paper_1909_08390_gb300", "csrc")
    subprocess.run(["g++", "-std=c++17"] + SAN +
                   ["-I", os.path.join(ROOT, "include"), "-I", csrc, "-I",
                    os.path.join(cuda, "include"), os.path.join(HERE, "host", "api_sanitize.cpp"),
                    os.path.join(csrc, "fdlb_api.cpp"), "-o", exe, "-L", lib64, "-lcudart",
                    "-Wl,-rpath," + lib64], check=True)
    assert "ok" in _run(exe)
