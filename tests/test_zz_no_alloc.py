"""fdlb_step_noalloc, the step for callers that cannot call cudaMalloc (for
example code inside a framework whose pool allocator owns all device memory,
or a loop that may not pay an allocation's latency and synchronisation).

It keeps its intermediate arrays in the library's static device scratch and
must give the same result as the regular context path.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it passes both alone and after the others.
"""
import numpy as np
import pytest

from paper_1909_08390_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def F():
    from paper_1909_08390_gb300 import build as B, fdlb
    B.build()
    fdlb.load()
    return fdlb


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("case", ["sod_1d_q8", "quadrant_2d_q53"])
def test_noalloc_matches_context_path_on_two_calls(F, case):
    import torch
    if case == "sod_1d_q8":
        wl = W.sod_1d()
        states, xs, ys = wl.states, wl.xsplit, 0.0
        steps = (25, 40)
    else:
        wl = W.quadrant_2d(W.BENCH_SEED, n=48, Q=5).replace(Qchi=3, ny=40, dt=2e-4)
        states, xs, ys = wl.states, 0.5, 0.5
        steps = (6, 9)
    grid = F.fdlb_grid(wl.d, wl.nx, wl.ny, wl.x0, wl.x1, wl.y0, wl.y1, wl.bc)
    stream = torch.cuda.current_stream()
    with F.Solver.from_workload(wl, stream=stream) as s:
        s.init_riemann(states, xs, ys)
        dev = torch.from_numpy(s.state()).to("cuda")  # caller-owned state
        for n in steps:  # two calls in a row: the scratch keeps the last call's contents
            F.fdlb_step_noalloc(grid, wl.Qphi, wl.Qchi, wl.gamma, wl.tau, wl.dt, dev, n,
                                stream=stream)
            s.step(n)
            torch.cuda.synchronize()
            want = s.state()
            got = dev.cpu().numpy()
            assert _rel(got, want) < TOL


def test_noalloc_rejects_problems_beyond_the_scratch(F):
    import torch
    # 5 arrays x 128 populations x 256^2 cells x 8 B = 335 MB > 64 MiB
    grid = F.fdlb_grid(2, 256, 256, 0.0, 1.0, 0.0, 1.0, 0)
    dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FdlbError) as e:
        F.fdlb_step_noalloc(grid, 8, 8, 1.4, 1e-6, 2.5e-5, dev, 1)
    assert e.value.code == F.FDLB_EINVAL
    assert "too large" in str(e.value)
