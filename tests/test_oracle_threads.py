"""The oracle's OpenMP loops leave its results unchanged: every output element
is computed by one thread with the same operations in the same order, so a
step on one thread and on several is bitwise the same (2-D seeded quadrants,
1-D shock tube, periodic and outlet ghosts, the moments and the initial
equilibria)."""
import numpy as np
import pytest

from paper_1909_08390_gb300 import workloads as W


@pytest.fixture
def threads(oracle):
    before = oracle.set_threads(0)
    yield oracle
    oracle.set_threads(before)


def _run(oracle, n, pr, F0, steps):
    assert oracle.set_threads(n) == n
    F = oracle.step(pr, F0, steps)
    return F, oracle.moments(pr, F)


@pytest.mark.parametrize("bc", [0, 1])
def test_threads_bitwise_2d(threads, bc):
    O = threads
    wl = W.quadrant_2d(W.BENCH_SEED)
    pr = O.Problem(d=2, nx=23, ny=17, x0=0.0, x1=1.0, y0=0.0, y1=0.7, bc=bc, Qphi=8, Qchi=8,
                   gamma=1.4, tau=1e-6, dt=2.5e-4)
    O.set_threads(1)
    F0 = O.init_states(pr, wl.states, 0.5, 0.35)
    O.set_threads(5)
    np.testing.assert_array_equal(F0, O.init_states(pr, wl.states, 0.5, 0.35))
    a, ma = _run(O, 1, pr, F0, 3)
    b, mb = _run(O, 5, pr, F0, 3)
    np.testing.assert_array_equal(a, b)
    for x, y in zip(ma, mb):
        np.testing.assert_array_equal(x, y)


def test_threads_bitwise_1d(threads):
    O = threads
    wl = W.sod_1d(nx=97)
    pr = O.Problem(d=1, nx=wl.nx, x0=wl.x0, x1=wl.x1, Qphi=5, Qchi=3, gamma=wl.gamma, tau=wl.tau,
                   dt=wl.dt)
    F0 = O.init_states(pr, wl.states, wl.xsplit)
    a, _ = _run(O, 1, pr, F0, 20)
    b, _ = _run(O, 3, pr, F0, 20)
    np.testing.assert_array_equal(a, b)
