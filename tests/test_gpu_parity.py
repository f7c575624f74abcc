"""GPU parity: the CUDA path (called through the C ABI) against the FP64 CPU
oracle, element by element, on the same seeded inputs.

Tolerance: 1e-12 relative, ||gpu - oracle||_inf / ||oracle||_inf per
distribution (phi block, chi block) and per moment field.  Both sides compute
in binary64 but round in different orders (fused multiply-adds, recurrence vs
literal double sum for the equilibria, different summation order of the
moments); the MP limiter is continuous in its inputs, so branch flips at ties
do not amplify those differences.
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


def problem(oracle, **kw):
    return oracle.Problem(**kw)


def solver(F, pr):
    return F.Solver(d=pr.d, nx=pr.nx, ny=pr.ny, x0=pr.x0, x1=pr.x1, y0=pr.y0, y1=pr.y1, bc=pr.bc,
                    Qphi=pr.Qphi, Qchi=pr.Qchi, gamma=pr.gamma, tau=pr.tau, dt=pr.dt)


def rel(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def compare_state(pr, got, want, tol=TOL):
    nphi = pr.Qphi ** pr.d
    r_phi = rel(got[:nphi], want[:nphi])
    r_chi = rel(got[nphi:], want[nphi:])
    assert r_phi < tol and r_chi < tol, (r_phi, r_chi)
    return max(r_phi, r_chi)


def compare_moments(oracle, pr, s, want_state, tol=TOL, tol_u=None, tol_T=None):
    """n and T relative to their max; u relative to max(|u|, 1) (the
    reference speed); tol_u and tol_T default to tol."""
    n, ux, uy, T = s.moments()
    on, oux, ouy, oT = oracle.moments(pr, want_state)
    tol_u = tol if tol_u is None else tol_u
    tol_T = tol if tol_T is None else tol_T
    assert rel(n, on) < tol, rel(n, on)
    assert rel(T, oT) < tol_T, rel(T, oT)
    eu = np.abs(ux - oux).max() / max(np.abs(oux).max(), 1.0)
    assert eu < tol_u, eu
    if pr.d == 2:
        ev = np.abs(uy - ouy).max() / max(np.abs(ouy).max(), 1.0)
        assert ev < tol_u, ev


def _sod_pair(oracle, F, nsteps):
    wl = W.sod_1d()
    pr = problem(oracle, d=1, nx=wl.nx, x0=wl.x0, x1=wl.x1, Qphi=8, Qchi=8, gamma=wl.gamma,
                 tau=wl.tau, dt=wl.dt)
    want = oracle.step(pr, oracle.init_states(pr, wl.states, wl.xsplit), nsteps)
    s = solver(F, pr)
    s.init_riemann(wl.states, wl.xsplit)
    s.step(nsteps)
    return pr, s, want


def test_sod_1d_q8_200_steps_all_fields(oracle, F):
    """1-D shock tube (Nx = 400, Q = 8, gamma = 7/5, tau = 1e-6, dt = 5e-5),
    200 steps: state, n, u and T all within 1e-12."""
    pr, s, want = _sod_pair(oracle, F, 200)
    with s:
        compare_state(pr, s.state(), want)
        compare_moments(oracle, pr, s, want)


def test_sod_1d_q8_full_run(oracle, F):
    """The same problem to t = 0.1 (2000 steps): distributions and n within
    1e-12.  The bounds on T and u are derived from the run's conditioning:
    differences in the last bit (rounding order of the equilibria, of the
    fused stage coefficients and of the stencil) act at every stage and grow
    linearly, about 4e-16 per step in the state; the largest T and u
    differences sit in the shock cell (n ~ 0.16), where the binary64 oracle
    itself is 2.4e-12 (T) and 8e-12 (u) away from its own extended-precision
    evaluation.  3e-12 (T) and 5e-12 (u) are allowed there."""
    pr, s, want = _sod_pair(oracle, F, W.sod_1d().nsteps)
    with s:
        compare_state(pr, s.state(), want)
        compare_moments(oracle, pr, s, want, tol_u=5e-12, tol_T=3e-12)


def test_init_is_the_oracle_equilibrium(oracle, F):
    for (d, Qp, Qc) in [(1, 8, 8), (1, 5, 3), (2, 8, 8), (2, 5, 3), (2, 3, 3)]:
        kw = dict(d=d, nx=23, ny=(19 if d == 2 else 1), x0=0.0, x1=1.0, y0=0.0, y1=1.0, Qphi=Qp,
                  Qchi=Qc, gamma=1.4, tau=1e-5, dt=1e-4)
        pr = problem(oracle, **kw)
        st = W.sod_1d().states if d == 1 else W.C11_STATES
        want = oracle.init_states(pr, st, 0.37, 0.61)
        with solver(F, pr) as s:
            s.init_riemann(st, 0.37, 0.61)
            compare_state(pr, s.state(), want, tol=1e-14)


def test_init_membrane_on_cell_centres(oracle, F):
    """Membranes through cell centres (odd cell counts, membrane at the domain
    centre) and on faces: every cell takes the same side as in the oracle, in
    single problems (1-D and 2-D) and in a batch, within 1e-14.  nx = 49, 103
    and 755 are lengths whose middle cell a rounded-centre comparison puts on
    the left."""
    st1 = [[0.884, -0.125, 0.164], [0.89, 0.267, 0.502]]
    for nx in (3, 49, 103, 755, 400):
        pr = problem(oracle, d=1, nx=nx, x0=-0.5, x1=0.5, Qphi=8, Qchi=8, gamma=1.2, tau=1e-6,
                     dt=2e-5)
        with solver(F, pr) as s:
            s.init_riemann(st1, 0.0)
            compare_state(pr, s.state(), oracle.init_states(pr, st1, 0.0), tol=1e-14)
    pr = problem(oracle, d=2, nx=37, ny=29, x0=0.0, x1=1.0, y0=0.0, y1=1.0, Qphi=5, Qchi=3,
                 gamma=1.4, tau=1e-5, dt=1e-4)
    with solver(F, pr) as s:
        s.init_riemann(W.C11_STATES, 0.5, 0.5)
        compare_state(pr, s.state(), oracle.init_states(pr, W.C11_STATES, 0.5, 0.5), tol=1e-14)
    nxs, gms = [49, 103, 755, 256, 107], [1.2, 1.4, 1.202, 1.6, 1.1]
    st = np.array([st1] * len(nxs))
    for prec in (0, 1):
        with F.BatchSolver(nxs, gms, tau=1e-6, dt=2e-5, precision=prec) as b:
            b.init_riemann(st)
            got = b.state()
        for j, (nx, g) in enumerate(zip(nxs, gms)):
            pr = problem(oracle, d=1, nx=nx, x0=-0.5, x1=0.5, Qphi=8, Qchi=8, gamma=g, tau=1e-6,
                         dt=2e-5)
            want = oracle.init_states(pr, st1, 0.0)
            # binary32 pairs hold about 48 bits of each population
            compare_state(pr, b.member(got, j), want, tol=1e-14 if prec == 0 else 1e-13)


@pytest.mark.parametrize("Q", [(8, 8), (5, 3), (3, 3)])
@pytest.mark.parametrize("nx", [1, 4, 7, 128, 129, 333])
@pytest.mark.parametrize("bc", [0, 1])
def test_1d_ragged_random_populations(oracle, F, Q, nx, bc):
    """Rough (random) populations exercise the limited MP branch everywhere;
    sizes below the halo, exactly one tile, one tile plus one, and a ragged
    multi-tile tail."""
    pr = problem(oracle, d=1, nx=nx, x0=0.0, x1=1.0, bc=bc, Qphi=Q[0], Qchi=Q[1], gamma=1.4,
                 tau=2e-4, dt=1e-4 * min(1.0, 64.0 / max(nx, 1)))
    F0 = W.random_populations(pr.shape, seed=nx + 7 * bc)
    want = oracle.step(pr, F0, 6)
    with solver(F, pr) as s:
        s.set_state(F0)
        s.step(6)
        compare_state(pr, s.state(), want)


@pytest.mark.parametrize("Q", [(8, 8), (5, 3), (3, 3)])
@pytest.mark.parametrize("shape", [(37, 29), (16, 16), (5, 3), (1, 1), (33, 17)])
@pytest.mark.parametrize("bc", [0, 1])
def test_2d_ragged_random_populations(oracle, F, Q, shape, bc):
    nx, ny = shape
    pr = problem(oracle, d=2, nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc=bc, Qphi=Q[0],
                 Qchi=Q[1], gamma=1.4, tau=1e-4, dt=2e-4 * 16.0 / max(nx, ny, 16))
    F0 = W.smooth_random_populations(pr.shape, seed=nx * ny + bc, amp=0.3)
    want = oracle.step(pr, F0, 4)
    with solver(F, pr) as s:
        s.set_state(F0)
        s.step(4)
        compare_state(pr, s.state(), want)


@pytest.mark.parametrize("seed", [1, 2])
def test_2d_quadrants_q8(oracle, F, seed):
    """Seeded four-quadrant Riemann problem (the 512^2 workload's states) on a
    ragged 48 x 40 grid, 30 steps."""
    wl = W.quadrant_2d(seed)
    pr = problem(oracle, d=2, nx=48, ny=40, x0=0.0, x1=1.0, y0=0.0, y1=1.0, Qphi=8, Qchi=8,
                 gamma=1.4, tau=wl.tau, dt=wl.dt * 8)
    want = oracle.step(pr, oracle.init_states(pr, wl.states, 0.5, 0.5), 30)
    with solver(F, pr) as s:
        s.init_riemann(wl.states, 0.5, 0.5)
        s.step(30)
        compare_state(pr, s.state(), want)
        compare_moments(oracle, pr, s, want)


def test_2d_paper_c11_q53(oracle, F):
    """Configuration 11 of Sec. V with the paper's lattice (Q = 5, 3; 34
    populations), tau = 1e-5, dt = 5e-4 on a 64 x 64 grid, 20 steps."""
    wl = W.lax_liu_2d(11, n=64)
    pr = problem(oracle, d=2, nx=64, ny=64, x0=wl.x0, x1=wl.x1, y0=wl.y0, y1=wl.y1, Qphi=5, Qchi=3,
                 gamma=1.4, tau=wl.tau, dt=wl.dt / 8)
    want = oracle.step(pr, oracle.init_states(pr, wl.states, 0.0, 0.0), 20)
    with solver(F, pr) as s:
        s.init_riemann(wl.states, 0.0, 0.0)
        s.step(20)
        compare_state(pr, s.state(), want)


def test_full_size_512_quadrants_one_step(oracle, F):
    """The benchmark workload itself (512 x 512, 8x8 velocities, 128
    populations, dt = 2.5e-5, tau = 1e-6), in the launch configuration the
    benchmark times: two full steps compared element by element."""
    wl = W.quadrant_2d(W.BENCH_SEED)
    pr = problem(oracle, d=2, nx=wl.nx, ny=wl.ny, x0=wl.x0, x1=wl.x1, y0=wl.y0, y1=wl.y1,
                 Qphi=8, Qchi=8, gamma=wl.gamma, tau=wl.tau, dt=wl.dt)
    want = oracle.step(pr, oracle.init_states(pr, wl.states, 0.5, 0.5), 2)
    with solver(F, pr) as s:
        s.init_riemann(wl.states, 0.5, 0.5)
        s.step(2)
        compare_state(pr, s.state(), want)


def test_conservation_periodic_gpu(oracle, F):
    pr = problem(oracle, d=2, nx=40, ny=24, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc=1, Qphi=8, Qchi=8,
                 gamma=1.4, tau=1e-5, dt=5e-4)
    F0 = W.smooth_random_populations(pr.shape, seed=3, amp=0.2)
    with solver(F, pr) as s:
        s.set_state(F0)
        n0, ux0, uy0, T0 = s.moments()
        s.step(200)
        n1, ux1, uy1, T1 = s.moments()
    tot = lambda n, ux, uy, T: np.array([n.sum(), (n * ux).sum(), (n * uy).sum(),
                                         (n * (ux * ux + uy * uy) + 5.0 * n * T).sum()])
    a, b = tot(n0, ux0, uy0, T0), tot(n1, ux1, uy1, T1)
    assert np.all(np.abs(a - b) <= 1e-12 * np.maximum(np.abs(a), 1.0)), (a, b)


def test_checkpoint_resume_is_bitwise(oracle, F):
    wl = W.sod_1d(nx=256)
    kw = dict(d=1, nx=256, x0=-0.5, x1=0.5, Qphi=8, Qchi=8, gamma=1.4, tau=1e-6, dt=5e-5)
    with F.Solver(**kw) as a, F.Solver(**kw) as b:
        a.init_riemann(wl.states, 0.0)
        a.step(100)
        b.init_riemann(wl.states, 0.0)
        b.step(40)
        ck = b.state()
        b.set_state(ck)
        b.step(60)
        assert np.array_equal(a.state(), b.state())


def test_invalid_state_reports_unstable(F):
    with F.Solver(d=1, nx=64, x0=0.0, x1=1.0, tau=1e-5, dt=1e-4) as s:
        s.set_state(-np.ones(s.shape))
        with pytest.raises(F.FdlbError) as e:
            s.step(1)
        assert e.value.code == F.FDLB_EUNSTABLE
        # a valid state clears the status
        s.init_riemann(W.sod_1d().states, 0.5)
        s.step(2)


def test_allocation_failure_reported(F):
    """A 20000^2 grid (4e8 cells, below the 2^30-cell limit) whose six
    binary64 population arrays need about 2.5 TB: the device allocation fails
    and fdlb_create returns FDLB_ENOMEM with no context."""
    g = F.fdlb_grid(2, 20000, 20000, 0.0, 1.0, 0.0, 1.0, F.FDLB_BC_OUTLET)
    with pytest.raises(F.FdlbError) as ei:
        F.fdlb_create(g, 8, 8, 1.4, 1e-6, 1e-7, None, F.FDLB_FP64, None)
    assert ei.value.code == F.FDLB_ENOMEM
    # the library and the device stay usable
    with F.Solver(d=1, nx=64) as s:
        s.init_riemann(W.sod_1d().states, 0.0)
        s.step(2)
