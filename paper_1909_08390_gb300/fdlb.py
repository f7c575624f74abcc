"""Thin ctypes binding of libfdlb.so (include/fdlb.h).

Argument marshalling only: every step of the method runs in the library's
sm_103a kernels.  The functions carry the C names (``fdlb_create``,
``fdlb_init_riemann``, ``fdlb_step``, ``fdlb_moments``, ``fdlb_get_state``,
``fdlb_set_state``, ``fdlb_destroy``, ...); ``Solver`` wraps a context for
convenience.  Host arrays are numpy arrays; device arrays are torch CUDA
tensors (PyTorch supplies device memory and streams).

There is no fallback: if ``libfdlb.so`` is missing or cannot be loaded,
``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfdlb.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "fdlb.h")

FDLB_OK = 0
FDLB_EINVAL = -1
FDLB_ECFL = -2
FDLB_ENOMEM = -3
FDLB_ECUDA = -4
FDLB_EUNSTABLE = -5
FDLB_ETIMEOUT = -6
FDLB_FP64 = 0
FDLB_MIXED = 1
FDLB_BC_OUTLET = 0
FDLB_BC_PERIODIC = 1
FDLB_TABLEAU_IMEX_SSP3_433 = 0
FDLB_TABLEAU_EXPLICIT_SSPRK3 = 1

_ERRNAMES = {0: "FDLB_OK", -1: "FDLB_EINVAL", -2: "FDLB_ECFL", -3: "FDLB_ENOMEM",
             -4: "FDLB_ECUDA", -5: "FDLB_EUNSTABLE", -6: "FDLB_ETIMEOUT"}


class fdlb_grid(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double), ("bc", ctypes.c_int)]


class fdlb_tableau(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int), ("At", ctypes.c_double * 16), ("A", ctypes.c_double * 16),
                ("wt", ctypes.c_double * 4), ("w", ctypes.c_double * 4)]


class FdlbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libfdlb.so (built by ``paper_1909_08390_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FdlbError(FDLB_ECUDA, f"{path} not built; run paper_1909_08390_gb300.build.build()")
    lib = ctypes.CDLL(path)
    lib.fdlb_create.argtypes = [ctypes.POINTER(fdlb_grid), ctypes.c_int, ctypes.c_int,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.POINTER(fdlb_tableau), ctypes.c_int, _vp, ctypes.POINTER(_vp)]
    lib.fdlb_create.restype = ctypes.c_int
    lib.fdlb_init_riemann.argtypes = [_vp, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    lib.fdlb_step.argtypes = [_vp, ctypes.c_int64]
    lib.fdlb_step_timed.argtypes = [_vp, ctypes.c_int64, _dp]
    lib.fdlb_moments.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_int]
    lib.fdlb_moments_adjoint.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    lib.fdlb_state_bytes.argtypes = [_vp]
    lib.fdlb_state_bytes.restype = ctypes.c_size_t
    lib.fdlb_get_state.argtypes = [_vp, _vp, ctypes.c_int]
    lib.fdlb_set_state.argtypes = [_vp, _vp, ctypes.c_int]
    lib.fdlb_npop.argtypes = [_vp]
    lib.fdlb_ncells.argtypes = [_vp]
    lib.fdlb_ncells.restype = ctypes.c_int64
    lib.fdlb_set_stream.argtypes = [_vp, _vp]
    lib.fdlb_launches_per_step.argtypes = [_vp]
    lib.fdlb_lattice_nodes.argtypes = [ctypes.c_int, _dp, _dp]
    _i64p = ctypes.POINTER(ctypes.c_int64)
    lib.fdlb_create_batch.argtypes = [ctypes.c_int, _i64p, _dp, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, _vp, ctypes.POINTER(_vp)]
    lib.fdlb_batch_init_riemann.argtypes = [_vp, _dp, _dp]
    lib.fdlb_batch_offsets.argtypes = [_vp, _i64p]
    lib.fdlb_batch_status.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint)]
    lib.fdlb_autotune.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int)]
    lib.fdlb_batch_set_tiling.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
    lib.fdlb_named_tableau.argtypes = [ctypes.c_int, ctypes.POINTER(fdlb_tableau)]
    lib.fdlb_init_fields.argtypes = [_vp, _vp, _vp, _vp]
    lib.fdlb_init_fields_adjoint.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _dp]
    lib.fdlb_forward_ckpt.argtypes = [_vp, ctypes.c_int64, ctypes.c_int, _vp]
    lib.fdlb_adjoint.argtypes = [_vp, ctypes.c_int64, ctypes.c_int, _vp, _vp, _dp]
    lib.fdlb_step_noalloc.argtypes = [ctypes.POINTER(fdlb_grid), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.POINTER(fdlb_tableau), _vp, ctypes.c_int64, _vp]
    lib.fdlb_measure_fp64_pipe.argtypes = [_vp, _dp, _dp]
    lib.fdlb_destroy.argtypes = [_vp]
    lib.fdlb_destroy.restype = None
    lib.fdlb_last_error.argtypes = [_vp]
    lib.fdlb_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def header_symbols(path: str = HEADER):
    """Names of the functions include/fdlb.h declares."""
    with open(path) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fdlb_[a-z_0-9]+)\s*\(", text)))


def _check(rc: int, ctx=None):
    if rc != FDLB_OK:
        msg = load().fdlb_last_error(ctx).decode()
        raise FdlbError(rc, msg)


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- functions with the C names -------------------------------------------

def fdlb_create(grid: fdlb_grid, Qphi: int, Qchi: int, gamma: float, tau: float, dt: float,
                tableau: fdlb_tableau | None = None, precision: int = FDLB_FP64, stream=None):
    lib = load()
    out = _vp()
    tab = ctypes.byref(tableau) if tableau is not None else None
    rc = lib.fdlb_create(ctypes.byref(grid), int(Qphi), int(Qchi), float(gamma), float(tau),
                         float(dt), tab, int(precision), _stream_handle(stream), ctypes.byref(out))
    _check(rc, None)
    return out


def fdlb_init_riemann(ctx, states, xsplit: float, ysplit: float = 0.0):
    st = np.ascontiguousarray(states, dtype=np.float64)
    _check(load().fdlb_init_riemann(ctx, st.ctypes.data_as(_dp), st.shape[0], float(xsplit),
                                    float(ysplit)), ctx)


def fdlb_step(ctx, nsteps: int):
    _check(load().fdlb_step(ctx, int(nsteps)), ctx)


def fdlb_step_timed(ctx, nsteps: int):
    """Returns the summed device ms of the stage-3, stage-4 and final kernels."""
    ms = (ctypes.c_double * 3)()
    _check(load().fdlb_step_timed(ctx, int(nsteps), ms), ctx)
    return [ms[0], ms[1], ms[2]]


def fdlb_moments(ctx, n, ux, uy, T, on_device: bool):
    ptr = (lambda a: None if a is None else (a.data_ptr() if on_device else a.ctypes.data))
    _check(load().fdlb_moments(ctx, ptr(n), ptr(ux), ptr(uy), ptr(T), int(on_device)), ctx)


def fdlb_moments_adjoint(ctx, nbar, uxbar, uybar, Tbar, Fbar):
    """Fbar = J^T (nbar, uxbar, uybar, Tbar) at the context's state (device
    float64 tensors; None for a zero adjoint)."""
    ptr = (lambda a: None if a is None else a.data_ptr())
    _check(load().fdlb_moments_adjoint(ctx, ptr(nbar), ptr(uxbar), ptr(uybar), ptr(Tbar),
                                       Fbar.data_ptr()), ctx)


def fdlb_state_bytes(ctx) -> int:
    return int(load().fdlb_state_bytes(ctx))


def fdlb_get_state(ctx, dst, on_device: bool):
    ptr = dst.data_ptr() if on_device else dst.ctypes.data
    _check(load().fdlb_get_state(ctx, ptr, int(on_device)), ctx)


def fdlb_set_state(ctx, src, on_device: bool):
    ptr = src.data_ptr() if on_device else src.ctypes.data
    _check(load().fdlb_set_state(ctx, ptr, int(on_device)), ctx)


def fdlb_npop(ctx) -> int:
    return int(load().fdlb_npop(ctx))


def fdlb_ncells(ctx) -> int:
    return int(load().fdlb_ncells(ctx))


def fdlb_set_stream(ctx, stream):
    _check(load().fdlb_set_stream(ctx, _stream_handle(stream)), ctx)


def fdlb_launches_per_step(ctx) -> int:
    return int(load().fdlb_launches_per_step(ctx))


def fdlb_lattice_nodes(Q: int):
    p = np.zeros(Q)
    w = np.zeros(Q)
    _check(load().fdlb_lattice_nodes(int(Q), p.ctypes.data_as(_dp), w.ctypes.data_as(_dp)), None)
    return p, w


def fdlb_step_noalloc(grid: fdlb_grid, Qphi: int, Qchi: int, gamma: float, tau: float,
                      dt: float, F, nsteps: int, tableau: fdlb_tableau | None = None,
                      stream=None):
    """Advance the device state F (a torch CUDA float64 tensor, updated in
    place) by nsteps steps with the library's static scratch (no allocation)."""
    tab = ctypes.byref(tableau) if tableau is not None else None
    rc = load().fdlb_step_noalloc(ctypes.byref(grid), int(Qphi), int(Qchi), float(gamma),
                                  float(tau), float(dt), tab, F.data_ptr(), int(nsteps),
                                  _stream_handle(stream))
    _check(rc, None)


def fdlb_create_batch(nx, gamma, x0: float, x1: float, Qphi: int, Qchi: int, tau: float,
                      dt: float, precision: int = FDLB_MIXED, stream=None):
    nxa = np.ascontiguousarray(nx, dtype=np.int64)
    ga = np.ascontiguousarray(gamma, dtype=np.float64)
    assert nxa.shape == ga.shape
    out = _vp()
    rc = load().fdlb_create_batch(int(nxa.size), nxa.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  ga.ctypes.data_as(_dp), float(x0), float(x1), int(Qphi), int(Qchi),
                                  float(tau), float(dt), int(precision), _stream_handle(stream),
                                  ctypes.byref(out))
    _check(rc, None)
    return out


def fdlb_batch_init_riemann(ctx, states, xsplit=None):
    st = np.ascontiguousarray(states, dtype=np.float64)
    xs = None if xsplit is None else np.ascontiguousarray(xsplit, dtype=np.float64)
    _check(load().fdlb_batch_init_riemann(ctx, st.ctypes.data_as(_dp),
                                          None if xs is None else xs.ctypes.data_as(_dp)), ctx)


def fdlb_batch_offsets(ctx, nprob: int):
    base = np.zeros(nprob, dtype=np.int64)
    _check(load().fdlb_batch_offsets(ctx, base.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), ctx)
    return base


def fdlb_batch_status(ctx, nprob: int):
    flags = np.zeros(nprob, dtype=np.uint32)
    _check(load().fdlb_batch_status(ctx, flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint))), ctx)
    return flags


def fdlb_autotune(ctx, trial_steps: int = 2):
    v, k = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().fdlb_autotune(ctx, int(trial_steps), ctypes.byref(v), ctypes.byref(k)), ctx)
    return v.value, k.value


def fdlb_batch_set_tiling(ctx, variant: int, ctas_per_sm: int):
    _check(load().fdlb_batch_set_tiling(ctx, int(variant), int(ctas_per_sm)), ctx)


def fdlb_init_fields(ctx, n, u, T):
    """F = equilibrium of the per-cell fields (torch CUDA float64 tensors)."""
    _check(load().fdlb_init_fields(ctx, n.data_ptr(), u.data_ptr(), T.data_ptr()), ctx)


def fdlb_init_fields_adjoint(ctx, Fbar, n, u, T, nbar, ubar, Tbar) -> float:
    dg = ctypes.c_double(0.0)
    _check(load().fdlb_init_fields_adjoint(ctx, Fbar.data_ptr(), n.data_ptr(), u.data_ptr(),
                                           T.data_ptr(), nbar.data_ptr(), ubar.data_ptr(),
                                           Tbar.data_ptr(), ctypes.byref(dg)), ctx)
    return dg.value


def fdlb_forward_ckpt(ctx, nsteps: int, every: int, ckpt):
    _check(load().fdlb_forward_ckpt(ctx, int(nsteps), int(every), ckpt.data_ptr()), ctx)


def fdlb_adjoint(ctx, nsteps: int, every: int, ckpt, Fbar):
    """Fbar (in: dL/dF(nsteps), out: dL/dF(0)); returns (dL/dgamma, dL/dtau) of the steps."""
    d = (ctypes.c_double * 2)()
    _check(load().fdlb_adjoint(ctx, int(nsteps), int(every), ckpt.data_ptr(), Fbar.data_ptr(), d),
           ctx)
    return d[0], d[1]


def fdlb_measure_fp64_pipe(stream=None):
    """Measured binary64 FMA rate of the current device: (DFMA/s, ms of the timed launch)."""
    r, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().fdlb_measure_fp64_pipe(_stream_handle(stream), ctypes.byref(r), ctypes.byref(ms)),
           None)
    return r.value, ms.value


def fdlb_destroy(ctx):
    if ctx:
        load().fdlb_destroy(ctx)


def fdlb_last_error(ctx=None) -> str:
    return load().fdlb_last_error(ctx).decode()


def fdlb_named_tableau(which: int) -> fdlb_tableau:
    t = fdlb_tableau()
    _check(load().fdlb_named_tableau(int(which), ctypes.byref(t)), None)
    return t


def tableau_dict(t: fdlb_tableau) -> dict:
    """The tableau as nested lists (At, A, wt, w), r x r."""
    r = t.r
    return {"At": [[t.At[i * r + j] for j in range(r)] for i in range(r)],
            "A": [[t.A[i * r + j] for j in range(r)] for i in range(r)],
            "wt": [t.wt[i] for i in range(r)], "w": [t.w[i] for i in range(r)]}


def make_tableau(At, A, wt, w) -> fdlb_tableau:
    t = fdlb_tableau()
    r = len(w)
    t.r = r
    for i in range(r):
        for j in range(r):
            t.At[i * r + j] = At[i][j]
            t.A[i * r + j] = A[i][j]
        t.wt[i] = wt[i]
        t.w[i] = w[i]
    return t


# ---- convenience wrapper ---------------------------------------------------

class Solver:
    """One library context.  ``Solver.from_workload(wl)`` builds it from a
    ``workloads.Workload``."""

    def __init__(self, d: int, nx: int, ny: int = 1, x0: float = -0.5, x1: float = 0.5,
                 y0: float = 0.0, y1: float = 1.0, bc: int = FDLB_BC_OUTLET, Qphi: int = 8,
                 Qchi: int = 8, gamma: float = 1.4, tau: float = 1e-6, dt: float = 5e-5,
                 tableau: fdlb_tableau | None = None, precision: int = FDLB_FP64, stream=None):
        g = fdlb_grid(d, nx, ny if d == 2 else 1, x0, x1, y0, y1, bc)
        self.d, self.nx, self.ny = d, nx, (ny if d == 2 else 1)
        self.ctx = fdlb_create(g, Qphi, Qchi, gamma, tau, dt, tableau, precision, stream)
        self.P = fdlb_npop(self.ctx)
        self.N = fdlb_ncells(self.ctx)
        self.precision = precision
        self.dtype = np.float64  # both precisions exchange the state as binary64

    @classmethod
    def from_workload(cls, wl, precision: int = FDLB_FP64, stream=None, **kw):
        args = dict(d=wl.d, nx=wl.nx, ny=wl.ny, x0=wl.x0, x1=wl.x1, y0=wl.y0, y1=wl.y1, bc=wl.bc,
                    Qphi=wl.Qphi, Qchi=wl.Qchi, gamma=wl.gamma, tau=wl.tau, dt=wl.dt)
        args.update(kw)
        return cls(precision=precision, stream=stream, **args)

    @property
    def shape(self):
        return (self.P, self.ny, self.nx) if self.d == 2 else (self.P, self.nx)

    def init_riemann(self, states, xsplit: float, ysplit: float = 0.0):
        fdlb_init_riemann(self.ctx, states, xsplit, ysplit)

    def step(self, nsteps: int = 1):
        fdlb_step(self.ctx, nsteps)

    def state(self) -> np.ndarray:
        """The populations as float64 (a FDLB_MIXED state's binary32 pairs
        hi + lo summed and rounded once)."""
        out = np.empty(self.shape, dtype=self.dtype)
        fdlb_get_state(self.ctx, out, False)
        return out

    def set_state(self, F):
        if hasattr(F, "data_ptr"):
            assert F.element_size() == np.dtype(self.dtype).itemsize
            fdlb_set_state(self.ctx, F, True)
        else:
            F = np.ascontiguousarray(F, dtype=self.dtype)
            assert F.size == self.P * self.N
            fdlb_set_state(self.ctx, F, False)

    def moments(self):
        sh = self.shape[1:]
        n, ux, T = (np.empty(sh) for _ in range(3))
        uy = np.empty(sh) if self.d == 2 else None
        fdlb_moments(self.ctx, n, ux, uy, T, False)
        return n, ux, uy, T

    def close(self):
        if self.ctx:
            fdlb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class BatchSolver(Solver):
    """Independent 1-D problems in one context (fdlb_create_batch)."""

    def __init__(self, nx, gamma, x0: float = -0.5, x1: float = 0.5, Qphi: int = 8, Qchi: int = 8,
                 tau: float = 1e-6, dt: float = 2e-5, precision: int = FDLB_MIXED, stream=None):
        self.d, self.ny = 1, 1
        self.nprob = len(nx)
        self.nxs = np.asarray(nx, dtype=np.int64)
        self.ctx = fdlb_create_batch(nx, gamma, x0, x1, Qphi, Qchi, tau, dt, precision, stream)
        self.P = fdlb_npop(self.ctx)
        self.N = fdlb_ncells(self.ctx)
        self.nx = self.N
        self.precision = precision
        self.dtype = np.float64  # both precisions exchange the state as binary64
        self.base = fdlb_batch_offsets(self.ctx, self.nprob)

    def init_riemann(self, states, xsplit=None):
        fdlb_batch_init_riemann(self.ctx, states, xsplit)

    def autotune(self, trial_steps: int = 2):
        return fdlb_autotune(self.ctx, trial_steps)

    def status(self):
        """Per-problem flags (bit 0: the problem went unstable)."""
        return fdlb_batch_status(self.ctx, self.nprob)

    def step(self, nsteps: int = 1, allow_unstable: bool = False):
        """Advance; with allow_unstable, a member that went unstable does not
        raise (check status())."""
        try:
            fdlb_step(self.ctx, nsteps)
        except FdlbError as e:
            if not (allow_unstable and e.code == FDLB_EUNSTABLE):
                raise

    def member(self, arr, i):
        """Slice of problem i from a concatenated per-cell array (last axis)."""
        return arr[..., self.base[i]:self.base[i] + self.nxs[i]]


# ---- differentiation (torch.autograd) --------------------------------------

def _field_context(spec, gamma: float, tau: float, n0, u0, T0):
    """A 1-D binary64 outlet context whose state is the equilibrium of the
    fields (n0, u0, T0) (CUDA float64 tensors of spec['nx'] cells)."""
    import torch
    Q = spec["Q"]
    Qphi, Qchi = Q if isinstance(Q, tuple) else (Q, Q)
    g = fdlb_grid(1, spec["nx"], 1, spec["x0"], spec["x1"], 0.0, 1.0, FDLB_BC_OUTLET)
    ctx = fdlb_create(g, Qphi, Qchi, float(gamma), float(tau), spec["dt"], None, FDLB_FP64,
                      torch.cuda.current_stream())
    try:
        fdlb_init_fields(ctx, *(t.detach().to(torch.float64).contiguous() for t in (n0, u0, T0)))
    except Exception:
        fdlb_destroy(ctx)
        raise
    return ctx, Qphi


def _density(ctx, nx: int, device):
    """The density of the context's state, from the library's moments kernel."""
    import torch
    n, u, T = (torch.empty(nx, dtype=torch.float64, device=device) for _ in range(3))
    fdlb_moments(ctx, n, u, None, T, True)
    return n


def density_forward(n0, u0, T0, gamma, tau, spec):
    """Final density after spec['nsteps'] steps from the equilibrium of the
    fields (no gradient; the plain fdlb_step path)."""
    import torch
    ctx, _ = _field_context(spec, gamma, tau, n0, u0, T0)
    try:
        fdlb_step(ctx, spec["nsteps"])
        n = _density(ctx, spec["nx"], n0.device)
        torch.cuda.current_stream().synchronize()
    finally:
        fdlb_destroy(ctx)
    return n


def _autograd_function():
    import torch

    class DensityRun(torch.autograd.Function):
        """Final density n(x) after nsteps IMEX steps of a 1-D binary64 problem
        started from the equilibrium of the fields (n0, u0, T0), as a
        differentiable function of the fields, gamma and tau.  Forward: the
        checkpointed run (fdlb_forward_ckpt, a state kept every `every`
        steps).  Backward: the library's hand-written discrete adjoint
        (fdlb_adjoint, then fdlb_init_fields_adjoint)."""

        @staticmethod
        def forward(fctx, n0, u0, T0, gamma, tau, spec):
            nsteps, every = spec["nsteps"], spec["every"]
            ctx, Qphi = _field_context(spec, gamma, tau, n0, u0, T0)
            try:
                P = fdlb_npop(ctx)
                ckpt = torch.empty((nsteps // every + 1, P, spec["nx"]), dtype=torch.float64,
                                   device=n0.device)
                fdlb_forward_ckpt(ctx, nsteps, every, ckpt)
                n = _density(ctx, spec["nx"], n0.device)
                torch.cuda.current_stream().synchronize()
            finally:
                fdlb_destroy(ctx)
            fctx.ckpt, fctx.spec, fctx.P = ckpt, spec, P
            fctx.gamma, fctx.tau = float(gamma), float(tau)
            fctx.save_for_backward(*(t.detach().to(torch.float64).contiguous() for t in (n0, u0, T0)))
            return n

        @staticmethod
        def backward(fctx, nbar):
            n0, u0, T0 = fctx.saved_tensors
            spec = fctx.spec
            Fbar = torch.empty((fctx.P, spec["nx"]), dtype=torch.float64, device=nbar.device)
            ctx, _ = _field_context(spec, fctx.gamma, fctx.tau, n0, u0, T0)
            try:
                # dLoss/dF(nsteps) from dLoss/dn: the library's transpose of
                # the moment map (n is linear in F, so the context's current
                # state does not enter)
                fdlb_moments_adjoint(ctx, nbar.to(torch.float64).contiguous(), None, None, None,
                                     Fbar)
                dg, dtau = fdlb_adjoint(ctx, spec["nsteps"], spec["every"], fctx.ckpt, Fbar)
                nb, ub, Tb = (torch.empty_like(n0) for _ in range(3))
                dg0 = fdlb_init_fields_adjoint(ctx, Fbar, n0, u0, T0, nb, ub, Tb)
                torch.cuda.current_stream().synchronize()
            finally:
                fdlb_destroy(ctx)
            fctx.ckpt = None
            dev = nbar.device
            return (nb, ub, Tb, torch.tensor(dg + dg0, dtype=torch.float64, device=dev),
                    torch.tensor(dtau, dtype=torch.float64, device=dev), None)

    return DensityRun


_DensityRun = None


def density_run(n0, u0, T0, gamma, tau, spec):
    """Differentiable final density (see DensityRun); spec holds nx, x0, x1,
    Q (int or (Qphi, Qchi)), dt, nsteps and every."""
    global _DensityRun
    if _DensityRun is None:
        _DensityRun = _autograd_function()
    return _DensityRun.apply(n0, u0, T0, gamma, tau, spec)


def blended_fields(params, nx: int, x0: float = -0.5, x1: float = 0.5, width: float = 0.05):
    """Initial fields (n, u, T = P/rho) of the blended two-state data (the
    seeded-input recipe of workloads.blend_states) as differentiable torch
    operations on params = (rhoL, uL, PL, rhoR, uR, PR)."""
    import torch
    from .workloads import blend_states, cell_centres
    x = torch.as_tensor(cell_centres(nx, x0, x1), dtype=torch.float64, device=params.device)
    rho, u, P = blend_states(params, x, width, torch.tanh)
    return rho, u, P / rho
