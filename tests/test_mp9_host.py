"""The CUDA path's MP-9 routine (fdlb_mp9.cuh: binary64 arithmetic, integer
comparisons on bit patterns, interface values from forward differences),
compiled for the host, against the oracle's literal Sec. IV formulas."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "host", "mp9_host.cpp")
HDR = os.path.join(os.path.dirname(HERE), "paper_1909_08390_gb300", "csrc", "fdlb_mp9.cuh")
LIB = os.path.join(HERE, "host", "_build", "libmp9host.so")


@pytest.fixture(scope="module")
def mp9():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(HDR)):
        tmp = LIB + f".{os.getpid()}"
        subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", SRC,
                        "-o", tmp], check=True)
        os.replace(tmp, LIB)
    lib = ctypes.CDLL(LIB)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.mp9_face.argtypes = [dp]
    lib.mp9_face.restype = ctypes.c_double
    lib.mp9_line.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
    lib.mp9_line_march8.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
    lib.mp9_face_f32.argtypes = [ctypes.POINTER(ctypes.c_float)]
    lib.mp9_face_f32.restype = ctypes.c_float
    lib.mp9_dm_bits.argtypes = [ctypes.c_double, ctypes.c_double]
    lib.mp9_dm_bits.restype = ctypes.c_longlong
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def windows(rng, n):
    kinds = []
    for _ in range(n):
        k = rng.integers(0, 6)
        if k == 0:
            v = rng.normal(size=9)
        elif k == 1:
            v = np.cumsum(np.abs(rng.normal(size=9)))
        elif k == 2:
            v = np.where(np.arange(9) < rng.integers(1, 9), 1.0, 0.125) + 1e-3 * rng.normal(size=9)
        elif k == 3:
            x = np.arange(9) - 4 + rng.uniform(-1, 1)
            v = -x * x * rng.uniform(0.1, 3)
        elif k == 4:
            v = np.full(9, rng.uniform(-2, 2))
            v[rng.integers(0, 9)] += rng.choice([0.0, 1e-12, -3.0])
        else:
            v = rng.integers(-3, 4, size=9).astype(float)
        kinds.append(v * rng.choice([1e-6, 1.0, 1e3]))
    return kinds


def test_face_matches_oracle(oracle, mp9):
    rng = np.random.default_rng(0)
    nlim = 0
    for v in windows(rng, 20000):
        want, lim = oracle.mp9_face(v)
        nlim += lim
        got = mp9.mp9_face(_p(np.ascontiguousarray(v)))
        scale = np.abs(v).max()
        assert abs(got - want) <= 4e-15 * max(scale, 1e-300), (v, got, want)
    assert nlim > 2000  # the limited branch is exercised


def test_binary32_face_matches_oracle(oracle, mp9):
    """The binary32 face of the mixed-precision path (bounds at twice their
    value, three-input min/max) against the oracle's binary64 Sec. IV
    formulas on the same binary32 windows: the limiter is continuous in its
    inputs, so the two agree to a few binary32 roundings of the window's
    scale, in both branches."""
    rng = np.random.default_rng(3)
    nlim = 0
    for v in windows(rng, 20000):
        v32 = np.ascontiguousarray(v, dtype=np.float32)
        want, lim = oracle.mp9_face(v32.astype(np.float64))
        nlim += lim
        got = mp9.mp9_face_f32(v32.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        scale = float(np.abs(v32).max())
        assert abs(got - want) <= 2e-6 * max(scale, 1e-30), (v32, got, want)
    assert nlim > 2000


def test_hand_examples(mp9):
    import json
    with open(os.path.join(HERE, "golden", "mp9_hand_examples.json")) as f:
        for e in json.load(f)["examples"]:
            got = mp9.mp9_face(_p(np.asarray(e["v"], dtype=float)))
            assert abs(got - e["face"]) < 1e-15, (e, got)


@pytest.mark.parametrize("sgn", [1, -1])
def test_line_march_matches_oracle_advection(oracle, mp9, sgn):
    """Marched interface values, in 1- and 8-interface segments, give the
    oracle's flux differences on random lines with outlet ghosts."""
    rng = np.random.default_rng(1 + (sgn > 0))
    for trial in range(50):
        n = 127
        F = np.cumsum(rng.normal(size=n)) * 0.1 + 2.0 if trial % 2 else rng.uniform(0.5, 1.5, size=n)
        ext = np.concatenate([np.full(5, F[0]), F, np.full(5, F[-1])])
        a = np.zeros(n + 1)
        b = np.zeros(n + 1)
        mp9.mp9_line(_p(ext), n, sgn, _p(a))
        mp9.mp9_line_march8(_p(ext), n, sgn, _p(b))
        np.testing.assert_array_equal(a, b)
        ds = 0.01
        p = 1.7 * sgn
        want = oracle.advect_line(F, p, ds, bc=0)
        got = p * (a[1:] - a[:-1]) / ds
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


def _minmod4_literal(*xs):
    """Sec. IV's four-argument minmod taken literally: the argument of
    smallest magnitude (the first of equal ones) if all four are nonzero and
    share a sign, else zero."""
    if all(x > 0 for x in xs) or all(x < 0 for x in xs):
        best = xs[0]
        for x in xs[1:]:
            if abs(x) < abs(best):
                best = x
        return best
    return 0.0


def _bits(x):
    return int(np.array(x, dtype=np.float64).view(np.int64))


def test_dm_one_operation_matches_four_argument_minmod(mp9):
    """The march forms DM = minmod4(4a - b, 4b - a, a, b) from one fma
    (the smaller-magnitude curvature m, the other M, and 4m - M): bitwise the
    literal minmod4, +0 included, on random pairs and on ties, signed zeros,
    equal magnitudes and the boundary 4|m| - |M| = |m|."""
    rng = np.random.default_rng(5)
    pairs = [(a, b) for a in (0.0, -0.0, 1.0, -1.0, 3.0, -3.0, 0.25, 4.0, 5e-324, -2.5e-300)
             for b in (0.0, -0.0, 1.0, -1.0, 3.0, -3.0, 0.75, 4.0, 1e300, -7.0)]
    pairs += [(x, 3.0 * x) for x in (1.0, -2.0, 0.1, 1e-200)]  # 4m - M = m
    pairs += [(3.0 * x, x) for x in (1.0, -2.0, 0.1, 1e-200)]
    pairs += [(x, x) for x in (1.0, -0.3)]
    for _ in range(20000):
        a, b = rng.normal(size=2) * rng.choice([1e-8, 1.0, 1e8], size=2)
        if rng.random() < 0.3:
            b = a * rng.choice([0.25, 0.26, 1.0, 2.9, 3.0, 3.1, 4.0, 5.0, -1.0])
        pairs.append((float(a), float(b)))
    for a, b in pairs:
        # 4a is exact here, so 4a - b rounds once, as fma(4, a, -b) does
        want = _minmod4_literal(4.0 * a - b, 4.0 * b - a, a, b)
        got = mp9.mp9_dm_bits(a, b)
        assert got == _bits(want if want != 0 else 0.0), (a, b, want)
