"""The mixed-precision kernels' binary32-pair arithmetic and equilibrium
factors, compiled for the host from their own source (the section of
csrc/fdlb_mixed.cu between the pair-arithmetic and equilibrium-factor
markers, with the CUDA intrinsics replaced by host operations rounded once
each, -ffp-contract=off), against extended-precision evaluations (C long
double via numpy.longdouble; 64-bit significands on x86-64).

* TwoSum pair addition and the fma-based pair product: within a few units of
  2^-48 relative to their exact results.
* The axis factors g_k = sum_l c_lk a_l(u, T) * scale of Eq. (gExpanded):
  a_0 = scale, a_1 = scale u, a_l = u a_{l-1} + (l-1)(T-1) a_{l-2}, and
  c_lk = w_k He_l(p_k)/l! as binary32 pairs, evaluated as in the kernels,
  for the (3, 5, 8)-point rules, over velocities and temperatures on both
  sides of the lattice's reference: the pair result is within 2e-13 of the
  sum of the terms' magnitudes.  A slip in the node pairing, in the mirror
  index of the odd part or in a sign of the recurrence fails it at O(1)."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "host", "pair_host.cpp")
MIXED = os.path.join(ROOT, "paper_1909_08390_gb300", "csrc", "fdlb_mixed.cu")
BUILD = os.path.join(HERE, "host", "_build")
LIB = os.path.join(BUILD, "libpairhost.so")
BEGIN = "// ---- binary32 pairs: x = hi + lo with about 48 significant bits"
END = "// Equilibrium factors of a cell (Eq. gExpanded)"
LD = np.longdouble


@pytest.fixture(scope="module")
def lib():
    if np.finfo(LD).nmant <= 52:
        pytest.skip("long double is binary64 on this host")
    os.makedirs(BUILD, exist_ok=True)
    text = open(MIXED).read()
    i, j = text.index(BEGIN), text.index(END)
    with open(os.path.join(BUILD, "pair_extract.inc"), "w") as f:
        f.write(text[i:j])
    tmp = LIB + f".{os.getpid()}"
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                    "-I", os.path.join(HERE, "host"), SRC, "-o", tmp], check=True)
    os.replace(tmp, LIB)
    L = ctypes.CDLL(LIB)
    fp = ctypes.POINTER(ctypes.c_float)
    L.host_axis_g_df.argtypes = [ctypes.c_int, fp, fp] + [ctypes.c_float] * 6 + [fp, fp]
    for name in ("host_df_mul", "host_df_add"):
        getattr(L, name).argtypes = [ctypes.c_float] * 4 + [fp, fp]
    return L


def split(x):
    """binary64 -> binary32 pair (hi rounded, lo the rounded residual)."""
    hi = np.float32(x)
    return hi, np.float32(np.float64(x) - np.float64(hi))


def pair_value(h, l):
    return LD(np.float64(h)) + LD(np.float64(l))


def test_pair_add_and_mul(lib):
    rng = np.random.default_rng(5)
    out_h, out_l = ctypes.c_float(), ctypes.c_float()
    for _ in range(3000):
        a, b = rng.normal() * 10.0 ** rng.integers(-3, 3), rng.normal() * 10.0 ** rng.integers(-3, 3)
        ah, al = split(a)
        bh, bl = split(b)
        A, B = pair_value(ah, al), pair_value(bh, bl)
        lib.host_df_mul(ah, al, bh, bl, ctypes.byref(out_h), ctypes.byref(out_l))
        r = pair_value(out_h.value, out_l.value)
        assert abs(r - A * B) <= LD(2.0) ** -46 * abs(A * B), (a, b)
        lib.host_df_add(ah, al, bh, bl, ctypes.byref(out_h), ctypes.byref(out_l))
        r = pair_value(out_h.value, out_l.value)
        assert abs(r - (A + B)) <= LD(2.0) ** -46 * (abs(A) + abs(B)), (a, b)


def _rule(Q):
    """Probabilists' Gauss-Hermite nodes and weights normalised to sum 1, and
    the table c_lk = w_k He_l(p_k)/l! as the library stores it ([l][k])."""
    p, w = np.polynomial.hermite_e.hermegauss(Q)
    w = w / w.sum()
    c = np.zeros((16, 16))
    for l in range(Q):
        coef = np.zeros(l + 1)
        coef[l] = 1.0
        c[l, :Q] = w * np.polynomial.hermite_e.hermeval(p, coef) / math.factorial(l)
    return c


@pytest.mark.parametrize("Q", [3, 5, 8])
def test_axis_factors_against_extended_precision(lib, Q):
    c = _rule(Q)
    ch = np.zeros(256, dtype=np.float32)
    cl = np.zeros(256, dtype=np.float32)
    for idx, v in enumerate(c.ravel()):
        ch[idx], cl[idx] = split(v)
    fp = ctypes.POINTER(ctypes.c_float)
    gh = np.zeros(16, dtype=np.float32)
    gl = np.zeros(16, dtype=np.float32)
    rng = np.random.default_rng(Q)
    worst = 0.0
    for _ in range(400):
        u = rng.uniform(-1.2, 1.2)
        T = rng.uniform(0.1, 3.0)
        s = rng.uniform(0.1, 2.0)
        (uh, ul), (Th, Tl), (sh, sl) = split(u), split(T), split(s)
        assert lib.host_axis_g_df(Q, ch.ctypes.data_as(fp), cl.ctypes.data_as(fp), uh, ul, Th, Tl,
                                  sh, sl, gh.ctypes.data_as(fp), gl.ctypes.data_as(fp)) == 0
        U, TT, S = pair_value(uh, ul), pair_value(Th, Tl), pair_value(sh, sl)
        a = [S, S * U]
        for l in range(2, Q):
            a.append(U * a[l - 1] + LD(l - 1) * (TT - 1) * a[l - 2])
        for k in range(Q):
            terms = [pair_value(ch[l * 16 + k], cl[l * 16 + k]) * a[l] for l in range(Q)]
            exact = sum(terms, LD(0))
            got = pair_value(gh[k], gl[k])
            scale = sum((abs(t) for t in terms), LD(0))
            err = float(abs(got - exact) / scale)
            worst = max(worst, err)
            assert err < 2e-13, (Q, k, u, T, s, err)
    print(f"Q = {Q}: worst pair error / sum of |terms| = {worst:.2e}")
