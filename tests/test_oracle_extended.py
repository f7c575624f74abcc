"""The binary64 oracle against its own source built in extended precision
(C long double: 64-bit significands on x86-64), on the 1-D shock tube to
t = 0.1 (2000 steps).

This pins the conditioning argument behind the bars of the GPU's 2000-step
Sod parity test (distributions and n 1e-12, T 3e-12, u 5e-12). Every
binary64 evaluation of the scheme that rounds in a different order than the
oracle carries an error of about the oracle's own. The oracle's error is its
difference from the extended-precision evaluation of the same operations,
and it is of that size in T and u (largest in the shock cell). So bars
tighter than a few times 1e-12 in T and u could not be met by any binary64
implementation with a different rounding order.

The extended build is the oracle's source with every `double` made
`long double` and <tgmath.h> making its math calls type-generic; nothing
else changes. Constants written as binary64 literals stay binary64-rounded
(relative 1e-17), far below what is measured here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1909_08390_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "host", "_build")
MAXR = 8
LD = ctypes.c_longdouble


class _CfgLD(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", LD), ("x1", LD), ("y0", LD), ("y1", LD),
        ("bc", ctypes.c_int), ("Qphi", ctypes.c_int), ("Qchi", ctypes.c_int),
        ("gamma", LD), ("tau", LD), ("dt", LD),
        ("r", ctypes.c_int),
        ("At", (LD * MAXR) * MAXR), ("A", (LD * MAXR) * MAXR),
        ("wt", LD * MAXR), ("w", LD * MAXR),
        ("alpha_mp", LD),
    ]


@pytest.fixture(scope="module")
def ext():
    if ctypes.sizeof(LD) <= 8 or np.finfo(np.longdouble).nmant <= 52:
        pytest.skip("long double is binary64 on this host")
    os.makedirs(BUILD, exist_ok=True)
    src = {}
    for name in ("fdlb_oracle.c", "fdlb_oracle.h"):
        with open(os.path.join(ROOT, "oracle", name)) as f:
            text = re.sub(r"(?<!long )\bdouble\b", "long double", f.read())
        if name.endswith(".c"):
            text = text.replace("#include <math.h>", "#include <math.h>\n#include <tgmath.h>", 1)
        src[name] = text
    for name, text in src.items():
        with open(os.path.join(BUILD, "ext_" + name), "w") as f:
            f.write(text.replace('#include "fdlb_oracle.h"', '#include "ext_fdlb_oracle.h"'))
    lib = os.path.join(BUILD, "libfdlb_oracle_ext.so")
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    os.path.join(BUILD, "ext_fdlb_oracle.c"), "-o", lib, "-lm"], check=True)
    L = ctypes.CDLL(lib)
    ldp = ctypes.POINTER(LD)
    L.orc_paper_tableau.argtypes = [ctypes.POINTER(_CfgLD)]
    L.orc_init_states.argtypes = [ctypes.POINTER(_CfgLD), ldp, ctypes.c_int, LD, LD, ldp]
    L.orc_step.argtypes = [ctypes.POINTER(_CfgLD), ldp, ctypes.c_int]
    L.orc_moments.argtypes = [ctypes.POINTER(_CfgLD), ldp, ldp, ldp, ldp, ldp]
    L.orc_npop.argtypes = [ctypes.POINTER(_CfgLD)]
    L.orc_set_threads.argtypes = [ctypes.c_int]
    return L


def test_oracle_against_its_extended_precision_build(oracle, ext):
    wl = W.sod_1d()
    c = _CfgLD()
    c.d, c.nx, c.ny = 1, wl.nx, 1
    c.x0, c.x1, c.y0, c.y1 = wl.x0, wl.x1, 0.0, 1.0
    c.bc, c.Qphi, c.Qchi = 0, 8, 8
    c.gamma, c.tau, c.dt = wl.gamma, wl.tau, wl.dt
    ext.orc_paper_tableau(ctypes.byref(c))
    c.alpha_mp = 4.0
    P = ext.orc_npop(ctypes.byref(c))
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(LD))
    st = np.ascontiguousarray(wl.states, dtype=np.longdouble)
    F = np.zeros((P, wl.nx), dtype=np.longdouble)
    ext.orc_set_threads(os.cpu_count() or 1)
    assert ext.orc_init_states(ctypes.byref(c), ptr(st), 2, wl.xsplit, 0.0, ptr(F)) == 0
    assert ext.orc_step(ctypes.byref(c), ptr(F), wl.nsteps) == 0
    m = [np.zeros(wl.nx, dtype=np.longdouble) for _ in range(4)]
    assert ext.orc_moments(ctypes.byref(c), ptr(F), ptr(m[0]), ptr(m[1]), None, ptr(m[3])) == 0

    pr = oracle.Problem(d=1, nx=wl.nx, x0=wl.x0, x1=wl.x1, Qphi=8, Qchi=8, gamma=wl.gamma,
                        tau=wl.tau, dt=wl.dt)
    G = oracle.step(pr, oracle.init_states(pr, wl.states, wl.xsplit), wl.nsteps)
    n, u, _, T = oracle.moments(pr, G)
    ref = lambda a: np.asarray(a, dtype=np.float64)
    rel = lambda a, b, floor=0.0: float(np.abs(a - b).max() / max(np.abs(b).max(), floor))
    e_state = float(np.abs(G - F).max() / np.abs(F).max())
    e_n, e_u, e_T = rel(n, ref(m[0])), rel(u, ref(m[1]), 1.0), rel(T, ref(m[3]))
    print(f"binary64 oracle vs its extended build after {wl.nsteps} steps: state {e_state:.2e}, "
          f"n {e_n:.2e}, u {e_u:.2e}, T {e_T:.2e}")
    # the extended build computes the same scheme: the two runs agree to
    # 1e-10 everywhere
    assert e_state < 1e-10 and e_n < 1e-10 and e_u < 1e-10 and e_T < 1e-10
    # the binary64 oracle's own error in T and u is of the size of the GPU
    # test's bars (3e-12, 5e-12), and its error in the state and n of the
    # 1e-12 bar
    assert e_T > 1e-12 and e_u > 2e-12, (e_T, e_u)
    assert e_state > 2e-13 and e_n > 1e-13, (e_state, e_n)
