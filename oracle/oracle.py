"""ctypes binding of the FP64 CPU oracle (``fdlb_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library and never imports the product package.

The oracle follows the paper section by section (see the header of
``fdlb_oracle.c`` for the mapping and for the readings of passages where the
paper is silent or garbled).  Arrays use the layout ``F[P][ny][nx]``,
``P = Qphi**d + Qchi**d``, phi populations first (``k = ky*Qphi + kx``), then
chi populations (``q = qy*Qchi + qx``), nodes in ascending order.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdlb_oracle.c")
_HDR = os.path.join(_HERE, "fdlb_oracle.h")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXQ = 16
MAXR = 8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction) into oracle/_build."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("bc", ctypes.c_int), ("Qphi", ctypes.c_int), ("Qchi", ctypes.c_int),
        ("gamma", ctypes.c_double), ("tau", ctypes.c_double), ("dt", ctypes.c_double),
        ("r", ctypes.c_int),
        ("At", (ctypes.c_double * MAXR) * MAXR), ("A", (ctypes.c_double * MAXR) * MAXR),
        ("wt", ctypes.c_double * MAXR), ("w", ctypes.c_double * MAXR),
        ("alpha_mp", ctypes.c_double),
    ]


_dp = ctypes.POINTER(ctypes.c_double)


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_gauss_hermite.argtypes = [ctypes.c_int, _dp, _dp]
            lib.orc_g_axis.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp]
            lib.orc_g_axis.restype = None
            lib.orc_he_values.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
            lib.orc_he_values.restype = None
            lib.orc_paper_tableau.argtypes = [ctypes.POINTER(_Cfg)]
            lib.orc_paper_tableau.restype = None
            lib.orc_npop.argtypes = [ctypes.POINTER(_Cfg)]
            lib.orc_equilibrium.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_double, _dp,
                                            ctypes.c_double, _dp]
            lib.orc_moments.argtypes = [ctypes.POINTER(_Cfg), _dp, _dp, _dp, _dp, _dp]
            lib.orc_mp9_face.argtypes = [_dp, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]
            lib.orc_mp9_face.restype = ctypes.c_double
            lib.orc_advect_line.argtypes = [_dp, ctypes.c_int, ctypes.c_long, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_int, ctypes.c_double, _dp,
                                            ctypes.c_long]
            lib.orc_advect_line.restype = None
            lib.orc_advect.argtypes = [ctypes.POINTER(_Cfg), _dp, _dp]
            lib.orc_init_states.argtypes = [ctypes.POINTER(_Cfg), _dp, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_double, _dp]
            lib.orc_init_fields.argtypes = [ctypes.POINTER(_Cfg), _dp, _dp, _dp, _dp, _dp]
            lib.orc_step.argtypes = [ctypes.POINTER(_Cfg), _dp, ctypes.c_int]
            lib.orc_riemann_exact.argtypes = [ctypes.c_double] * 7 + [_dp, ctypes.c_int, _dp, _dp,
                                                                     _dp, _dp, _dp]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc}")


@dataclasses.dataclass
class Problem:
    """Parameters of one run (Sec. II-V).  tau <= 0 switches collisions off."""
    d: int = 1
    nx: int = 400
    ny: int = 1
    x0: float = -0.5
    x1: float = 0.5
    y0: float = 0.0
    y1: float = 1.0
    bc: int = 0              # 0 outlet (zero-gradient ghosts), 1 periodic
    Qphi: int = 8
    Qchi: int = 8
    gamma: float = 1.4
    tau: float = 1e-6
    dt: float = 5e-5
    tableau: dict | None = None   # None: IMEX-SSP3(4,3,3) of Table I
    alpha_mp: float = 4.0

    def cfg(self) -> _Cfg:
        c = _Cfg()
        c.d, c.nx, c.ny = self.d, self.nx, (self.ny if self.d == 2 else 1)
        c.x0, c.x1, c.y0, c.y1 = self.x0, self.x1, self.y0, self.y1
        c.bc, c.Qphi, c.Qchi = self.bc, self.Qphi, self.Qchi
        c.gamma, c.tau, c.dt = self.gamma, self.tau, self.dt
        _lib_handle().orc_paper_tableau(ctypes.byref(c))
        if self.tableau is not None:
            t = self.tableau
            r = len(t["w"])
            c.r = r
            for i in range(MAXR):
                for j in range(MAXR):
                    c.At[i][j] = t["At"][i][j] if i < r and j < r else 0.0
                    c.A[i][j] = t["A"][i][j] if i < r and j < r else 0.0
            for i in range(MAXR):
                c.wt[i] = t["wt"][i] if i < r else 0.0
                c.w[i] = t["w"][i] if i < r else 0.0
        c.alpha_mp = self.alpha_mp
        return c

    @property
    def ncell(self) -> int:
        return self.nx * (self.ny if self.d == 2 else 1)

    @property
    def npop(self) -> int:
        return self.Qphi ** self.d + self.Qchi ** self.d

    @property
    def shape(self):
        return (self.npop, self.ny, self.nx) if self.d == 2 else (self.npop, self.nx)


def paper_tableau() -> dict:
    c = _Cfg()
    _lib_handle().orc_paper_tableau(ctypes.byref(c))
    r = c.r
    return {
        "At": [[c.At[i][j] for j in range(r)] for i in range(r)],
        "A": [[c.A[i][j] for j in range(r)] for i in range(r)],
        "wt": [c.wt[i] for i in range(r)],
        "w": [c.w[i] for i in range(r)],
    }


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's OpenMP loops (n > 0 sets, n <= 0 keeps); returns
    the count in use.  The results are bitwise the same for any count."""
    return int(_lib_handle().orc_set_threads(int(n)))


def gauss_hermite(Q: int):
    p = np.zeros(Q)
    w = np.zeros(Q)
    _check(_lib_handle().orc_gauss_hermite(Q, _ptr(p), _ptr(w)), "gauss_hermite")
    return p, w


def he_values(Q: int, x: float) -> np.ndarray:
    out = np.zeros(Q)
    _lib_handle().orc_he_values(Q, float(x), _ptr(out))
    return out


def g_axis(Q: int, u: float, T: float) -> np.ndarray:
    p, w = gauss_hermite(Q)
    g = np.zeros(Q)
    _lib_handle().orc_g_axis(Q, _ptr(p), _ptr(w), float(u), float(T), _ptr(g))
    return g


def equilibrium(pr: Problem, n: float, u, T: float) -> np.ndarray:
    c = pr.cfg()
    uu = np.zeros(2)
    uu[: len(np.atleast_1d(u))] = np.atleast_1d(u)
    out = np.zeros(pr.npop)
    _check(_lib_handle().orc_equilibrium(ctypes.byref(c), float(n), _ptr(uu), float(T), _ptr(out)),
           "equilibrium")
    return out


def moments(pr: Problem, F: np.ndarray):
    """(n, ux, uy, T) per cell, Eq. (Moments_discrete); uy is None in 1-D."""
    c = pr.cfg()
    F = np.ascontiguousarray(F, dtype=np.float64)
    N = pr.ncell
    n, ux, T = np.zeros(N), np.zeros(N), np.zeros(N)
    uy = np.zeros(N) if pr.d == 2 else None
    rc = _lib_handle().orc_moments(ctypes.byref(c), _ptr(F), _ptr(n), _ptr(ux),
                                   _ptr(uy) if uy is not None else None, _ptr(T))
    _check(rc, "moments")
    sh = F.shape[1:]
    return (n.reshape(sh), ux.reshape(sh), None if uy is None else uy.reshape(sh), T.reshape(sh))


def mp9_face(v, alpha_mp: float = 4.0):
    """Interface value F_{s+1/2} for p > 0 from v = F_{s-4..s+4}; returns (value, limited)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    assert v.shape == (9,)
    lim = ctypes.c_int(0)
    val = _lib_handle().orc_mp9_face(_ptr(v), float(alpha_mp), ctypes.byref(lim))
    return val, bool(lim.value)


def advect_line(F, p: float, ds: float, bc: int = 0, alpha_mp: float = 4.0) -> np.ndarray:
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros_like(F)
    _lib_handle().orc_advect_line(_ptr(F), F.size, 1, float(p), float(ds), int(bc),
                                  float(alpha_mp), _ptr(out), 1)
    return out


def advect(pr: Problem, F: np.ndarray) -> np.ndarray:
    c = pr.cfg()
    F = np.ascontiguousarray(F, dtype=np.float64)
    LF = np.zeros_like(F)
    _check(_lib_handle().orc_advect(ctypes.byref(c), _ptr(F), _ptr(LF)), "advect")
    return LF


def init_states(pr: Problem, states, xsplit: float, ysplit: float = 0.5) -> np.ndarray:
    """Piecewise-constant Riemann data: 1-D states[2][(rho,u,P)],
    2-D states[4][(rho,ux,uy,P)] for quadrants 1..4."""
    c = pr.cfg()
    st = np.ascontiguousarray(states, dtype=np.float64)
    F = np.zeros(pr.shape)
    rc = _lib_handle().orc_init_states(ctypes.byref(c), _ptr(st), st.shape[0], float(xsplit),
                                       float(ysplit), _ptr(F))
    _check(rc, "init_states")
    return F


def init_fields(pr: Problem, rho, ux, uy, T) -> np.ndarray:
    c = pr.cfg()
    cast = lambda a: np.ascontiguousarray(np.broadcast_to(a, pr.shape[1:]), dtype=np.float64)
    rho, ux, T = cast(rho), cast(ux), cast(T)
    uy = cast(uy) if pr.d == 2 else None
    F = np.zeros(pr.shape)
    rc = _lib_handle().orc_init_fields(ctypes.byref(c), _ptr(rho), _ptr(ux),
                                       _ptr(uy) if uy is not None else None, _ptr(T), _ptr(F))
    _check(rc, "init_fields")
    return F


def step(pr: Problem, F: np.ndarray, nsteps: int = 1) -> np.ndarray:
    """Advance F by nsteps IMEX steps (Eq. IMEX); returns a new array."""
    c = pr.cfg()
    G = np.array(F, dtype=np.float64, order="C", copy=True)
    _check(_lib_handle().orc_step(ctypes.byref(c), _ptr(G), int(nsteps)), "step")
    return G


def riemann_exact(left, right, gamma: float, xi):
    """Exact Euler Riemann solution sampled at xi = x/t; left/right = (rho, u, p).
    Returns (rho, u, p, pstar, ustar)."""
    xi = np.ascontiguousarray(np.atleast_1d(xi), dtype=np.float64)
    rho, u, p = np.zeros_like(xi), np.zeros_like(xi), np.zeros_like(xi)
    ps, us = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = _lib_handle().orc_riemann_exact(*map(float, left), *map(float, right), float(gamma),
                                         _ptr(xi), xi.size, _ptr(rho), _ptr(u), _ptr(p),
                                         ctypes.cast(ctypes.pointer(ps), _dp),
                                         ctypes.cast(ctypes.pointer(us), _dp))
    _check(rc, "riemann_exact")
    return rho, u, p, ps.value, us.value
