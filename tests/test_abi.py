"""The C-ABI library loads, exports every symbol include/fdlb.h declares, and
rejects bad arguments before touching the GPU (no compute calls here)."""
import ctypes
import subprocess

import pytest

from paper_1909_08390_gb300 import fdlb
from paper_1909_08390_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return fdlb.load()


def test_header_declares_the_boundary():
    names = fdlb.header_symbols()
    for want in ("fdlb_create", "fdlb_init_riemann", "fdlb_step", "fdlb_moments", "fdlb_destroy",
                 "fdlb_get_state", "fdlb_set_state", "fdlb_last_error"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in fdlb.header_symbols() if n not in exported]
    assert not missing, missing
    for n in fdlb.header_symbols():
        assert hasattr(lib, n)


def _grid(**kw):
    g = dict(d=1, nx=64, ny=1, x0=-0.5, x1=0.5, y0=0.0, y1=1.0, bc=0)
    g.update(kw)
    return fdlb.fdlb_grid(g["d"], g["nx"], g["ny"], g["x0"], g["x1"], g["y0"], g["y1"], g["bc"])


@pytest.mark.parametrize("kw,args,code", [
    (dict(d=3), (8, 8, 1.4, 1e-6, 1e-5), fdlb.FDLB_EINVAL),
    (dict(nx=0), (8, 8, 1.4, 1e-6, 1e-5), fdlb.FDLB_EINVAL),
    (dict(x1=-0.5), (8, 8, 1.4, 1e-6, 1e-5), fdlb.FDLB_EINVAL),
    (dict(bc=7), (8, 8, 1.4, 1e-6, 1e-5), fdlb.FDLB_EINVAL),
    (dict(), (7, 7, 1.4, 1e-6, 1e-5), fdlb.FDLB_EINVAL),         # lattice not compiled
    (dict(), (8, 8, 1.0, 1e-6, 1e-5), fdlb.FDLB_EINVAL),         # gamma <= 1
    (dict(d=2, ny=8), (8, 8, 2.5, 1e-6, 1e-5), fdlb.FDLB_EINVAL),  # D+K-d < 0
    (dict(), (8, 8, 1.4, 0.0, 1e-5), fdlb.FDLB_EINVAL),          # tau
    (dict(), (8, 8, 1.4, 1e-6, -1.0), fdlb.FDLB_EINVAL),         # dt
    (dict(nx=400), (8, 8, 1.4, 1e-6, 1e-3), fdlb.FDLB_ECFL),     # 4.14*1e-3*400 > 1
    (dict(d=2, nx=65536, ny=65536), (8, 8, 1.4, 1e-6, 1e-8), fdlb.FDLB_EINVAL),  # 2^32 cells
])
def test_create_rejects_bad_arguments(lib, kw, args, code):
    out = ctypes.c_void_p()
    g = _grid(**kw)
    rc = lib.fdlb_create(ctypes.byref(g), args[0], args[1], args[2], args[3], args[4], None, 0,
                         None, ctypes.byref(out))
    assert rc == code, fdlb.fdlb_last_error(None)
    assert not out.value
    assert fdlb.fdlb_last_error(None) != "no error"


def test_create_rejects_unsupported_tableau(lib):
    # an advected first stage cannot be fused
    t = fdlb.make_tableau([[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [0, .25, .25, 0]],
                          [[.5, 0, 0, 0], [0, .5, 0, 0], [0, 0, .5, 0], [0, 0, 0, .5]],
                          [0, 1 / 6, 1 / 6, 2 / 3], [0, 1 / 6, 1 / 6, 2 / 3])
    out = ctypes.c_void_p()
    g = _grid()
    rc = lib.fdlb_create(ctypes.byref(g), 8, 8, 1.4, 1e-6, 1e-5, ctypes.byref(t), 0, None,
                         ctypes.byref(out))
    assert rc == fdlb.FDLB_EINVAL
    assert "tableau" in fdlb.fdlb_last_error(None)


def test_null_context_calls_fail_cleanly(lib):
    assert lib.fdlb_measure_fp64_pipe(None, None, None) == fdlb.FDLB_EINVAL
    assert lib.fdlb_step(None, 1) == fdlb.FDLB_EINVAL
    assert lib.fdlb_init_riemann(None, None, 2, 0.0, 0.0) == fdlb.FDLB_EINVAL
    assert lib.fdlb_state_bytes(None) == 0
    lib.fdlb_destroy(None)


@pytest.mark.parametrize("Q", [1, 2, 3, 4, 5, 6, 8, 10, 12, 16])
def test_library_lattice_nodes(lib, Q):
    """The library's Gauss-Hermite rule (host code, no GPU): numpy's rule, and
    exact antisymmetry of the nodes."""
    import numpy as np
    p, w = fdlb.fdlb_lattice_nodes(Q)
    pn, wn = np.polynomial.hermite_e.hermegauss(Q)
    np.testing.assert_allclose(p, pn, rtol=0, atol=2e-13)
    np.testing.assert_allclose(w, wn / np.sqrt(2 * np.pi), rtol=1e-11)
    np.testing.assert_array_equal(p, -p[::-1])


def test_named_tableaux(lib):
    """fdlb_named_tableau: Table I as printed, and the explicit comparator
    (Shu-Osher SSP-RK3 on the whole right-hand side) with its order
    conditions and stability polynomial."""
    import json
    import os

    import numpy as np

    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")) as fh:
        gold = json.load(fh)["tableau"]
    imex = fdlb.tableau_dict(fdlb.fdlb_named_tableau(fdlb.FDLB_TABLEAU_IMEX_SSP3_433))
    al, be, et = gold["alpha"], gold["beta"], gold["eta"]
    assert imex["At"] == gold["At"] and imex["wt"] == gold["wt"] and imex["w"] == gold["w"]
    A = np.array(imex["A"])
    want = np.array([[al, 0, 0, 0], [-al, al, 0, 0], [0, 1 - al, al, 0],
                     [be, et, 0.5 - be - et - al, al]])
    assert np.array_equal(A, want)

    ex = fdlb.tableau_dict(fdlb.fdlb_named_tableau(fdlb.FDLB_TABLEAU_EXPLICIT_SSPRK3))
    assert ex["At"] == ex["A"] and ex["wt"] == ex["w"]
    A, b = np.array(ex["A"]), np.array(ex["w"])
    assert np.all(np.triu(A) == 0)  # explicit: strictly lower triangular
    assert np.all(A[:, 0] == 0) and b[0] == 0 and np.all(A[1] == 0)  # the fused kernels' form
    c = A.sum(1)
    for got, exact in ((b.sum(), 1.0), (b @ c, 0.5), (b @ c ** 2, 1 / 3), (b @ A @ c, 1 / 6)):
        assert abs(got - exact) < 1e-15
    # stability function 1 + z b^T (I - zA)^-1 1 = 1 + z + z^2/2 + z^3/6 (order 3, 3 stages)
    for z in (-0.5, -1.0, -2.5, 0.3):
        R = 1 + z * b @ np.linalg.solve(np.eye(4) - z * A, np.ones(4))
        assert abs(R - (1 + z + z * z / 2 + z ** 3 / 6)) < 1e-14
    with pytest.raises(fdlb.FdlbError):
        fdlb.fdlb_named_tableau(7)
