"""The fully explicit comparator and the paper's own runs (Sec. V, Sec. VI).

* The explicit SSP-RK3 tableau (fdlb_named_tableau) runs through the same fused
  stage kernels; the GPU matches the oracle driven by the same tableau to
  1e-12 relative, and the scheme is unstable beyond dt/tau of about 2.5.
* Sec. VI's claim: the IMEX step at dt/tau = 50 reaches the explicit scheme's
  accuracy at dt/tau = 1 (50 times fewer steps), on the paper's shock tube.
* Fig. 1(a)/(b) sweeps and the 2-D configurations 11 and 12 of Fig. 2 as
  workloads, with what the paper states about them.
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


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def explicit(F):
    return F.fdlb_named_tableau(F.FDLB_TABLEAU_EXPLICIT_SSPRK3)


def run_sod(F, wl, tableau=None, nsteps=None):
    with F.Solver.from_workload(wl, tableau=tableau) as s:
        s.init_riemann(wl.states, wl.xsplit)
        s.step(wl.nsteps if nsteps is None else nsteps)
        return s.state(), s.moments()


def l1_density(oracle, wl, n):
    x = W.cell_centres(wl.nx, wl.x0, wl.x1)
    t = wl.nsteps * wl.dt
    rho = oracle.riemann_exact(wl.states[0], wl.states[1], wl.gamma, (x - wl.xsplit) / t)[0]
    return float(np.abs(n - rho).sum() * (wl.x1 - wl.x0) / wl.nx)


@pytest.mark.parametrize("Q", [(5, 3), (8, 8)])
def test_explicit_tableau_parity_1d(F, oracle, Q):
    """Sod, 200 nodes, tau = dt = 1e-5, 300 explicit steps: GPU vs oracle."""
    wl = W.sod_paper(S=200, dt=1e-5, Qphi=Q[0], Qchi=Q[1])
    tab = explicit(F)
    pr = oracle.Problem(d=1, nx=wl.nx, x0=wl.x0, x1=wl.x1, Qphi=Q[0], Qchi=Q[1], gamma=wl.gamma,
                        tau=wl.tau, dt=wl.dt, tableau=F.tableau_dict(tab))
    want = oracle.step(pr, oracle.init_states(pr, wl.states, wl.xsplit), 300)
    got, _ = run_sod(F, wl, tab, 300)
    nphi = Q[0]
    assert rel(got[:nphi], want[:nphi]) < TOL and rel(got[nphi:], want[nphi:]) < TOL


def test_explicit_tableau_parity_2d(F, oracle):
    """Seeded four-quadrant states on 37 x 29 cells, (5, 3) lattice, 30 steps."""
    wl = W.quadrant_2d(W.BENCH_SEED)
    tab = explicit(F)
    nx, ny, dt = 37, 29, 2e-4
    pr = oracle.Problem(d=2, nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, Qphi=5, Qchi=3,
                        gamma=1.4, tau=2e-4, dt=dt, tableau=F.tableau_dict(tab))
    want = oracle.step(pr, oracle.init_states(pr, wl.states, 0.5, 0.5), 30)
    with F.Solver(d=2, nx=nx, ny=ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, Qphi=5, Qchi=3, gamma=1.4,
                  tau=2e-4, dt=dt, tableau=tab) as s:
        s.init_riemann(wl.states, 0.5, 0.5)
        s.step(30)
        got = s.state()
    assert rel(got[:25], want[:25]) < TOL and rel(got[25:], want[25:]) < TOL


def test_explicit_scheme_unstable_beyond_its_limit(F):
    """dt/tau = 5 (|R(-5)| = 12.3): the non-equilibrium part grows until a
    cell's moments are invalid and the step reports FDLB_EUNSTABLE; the IMEX
    tableau at dt/tau = 50 on the same problem stays valid, as does the
    explicit one at dt/tau = 2."""
    wl = W.sod_paper(S=400, dt=5e-5)
    with F.Solver.from_workload(wl, tau=1e-5, tableau=explicit(F)) as s:
        s.init_riemann(wl.states, wl.xsplit)
        with pytest.raises(F.FdlbError) as ei:
            s.step(3000)
        assert ei.value.code == F.FDLB_EUNSTABLE
    with F.Solver.from_workload(wl, tau=2.5e-5, tableau=explicit(F)) as s:
        s.init_riemann(wl.states, wl.xsplit)
        s.step(3000)
    wl50 = W.sod_paper(S=400, dt=5e-4)
    run_sod(F, wl50)


def test_imex_fifty_fold_step_matches_explicit_accuracy(F, oracle):
    """Sec. VI: dt/tau = 50 with IMEX (300 steps to t = 0.15) against the
    explicit comparator at dt = tau (15000 steps), Q = (5, 3), 400 nodes.
    Both approximate the same viscous solution; their L1 density errors
    against the inviscid exact solution agree within 2 % (measured 0.3 %),
    and the two profiles differ by less than 5e-3 anywhere (measured 6.5e-4,
    in the shock and contact cells)."""
    imex = W.sod_paper(S=400, dt=5e-4)
    expl = W.sod_paper(S=400, dt=1e-5)
    assert expl.nsteps == 50 * imex.nsteps
    _, (n_i, _, _, _) = run_sod(F, imex)
    _, (n_e, _, _, _) = run_sod(F, expl, explicit(F))
    e_i, e_e = l1_density(oracle, imex, n_i), l1_density(oracle, expl, n_e)
    print(f"L1(rho): IMEX dt/tau=50 {e_i:.4e}, explicit dt/tau=1 {e_e:.4e}, "
          f"max |diff| {np.abs(n_i - n_e).max():.3e}")
    assert abs(e_i - e_e) <= 0.02 * e_e
    assert np.abs(n_i - n_e).max() < 5e-3


def test_fig1a_resolution_sweep(F, oracle):
    """Fig. 1(a): dt = 1e-5, S = 200 ... 3200.  The L1 density error against
    the inviscid solution falls with S while numerical dissipation dominates;
    at S = 3200 the physical dissipation of tau = 1e-5 sets the floor."""
    errs = []
    for S in W.FIG1A_S:
        wl = W.sod_paper(S=S, dt=W.FIG1A_DT)
        _, (n, _, _, _) = run_sod(F, wl)
        errs.append(l1_density(oracle, wl, n))
    print("Fig. 1(a) L1(rho):", dict(zip(W.FIG1A_S, np.round(errs, 6))))
    assert all(b < a for a, b in zip(errs[:4], errs[1:4]))
    assert errs[4] < errs[0]


def test_fig1b_time_step_sweep(F, oracle):
    """Fig. 1(b): S = 400, dt = 1e-3 ... 1e-5.  dt = 1e-3 puts the fastest
    (5, 3) node at CFL 1.14 > 1, which the library refuses (FDLB_ECFL); the
    paper shows that run with strong oscillations.  The other steps give the
    same L1 density error within 2 % (measured 0.4 %), and dt = 5e-4 agrees
    with dt = 1e-5 to within 5e-3 in every cell."""
    errs, prof = {}, {}
    for dt in W.FIG1B_DT:
        wl = W.sod_paper(S=W.FIG1B_S, dt=dt)
        if dt == 1e-3:
            with pytest.raises(F.FdlbError) as ei:
                run_sod(F, wl)
            assert ei.value.code == F.FDLB_ECFL
            continue
        _, (n, _, _, _) = run_sod(F, wl)
        errs[dt], prof[dt] = l1_density(oracle, wl, n), n
    print("Fig. 1(b) L1(rho):", {k: round(v, 6) for k, v in errs.items()})
    v = np.array(list(errs.values()))
    print(f"max |rho(5e-4) - rho(1e-5)| = {np.abs(prof[5e-4] - prof[1e-5]).max():.3e}")
    assert v.max() <= 1.02 * v.min()
    assert np.abs(prof[5e-4] - prof[1e-5]).max() < 5e-3


@pytest.mark.parametrize("config,rho_range", [(11, (0.52, 1.231)), (12, (0.53, 1.74))])
def test_lax_liu_configurations(F, config, rho_range):
    """Fig. 2: 400 x 400 nodes, Q = (5, 3) (34 populations), tau = 1e-5,
    dt = 5e-4, C11 to t = 0.3 and C12 to t = 0.25.  The paper's contour
    levels run from rho_min to rho_max; the computed density spans that range
    to within 0.015 at the low end and 1.5 % at the high end (measured:
    C11 [0.528, 1.2306], C12 [0.5313, 1.7318]; a weak pin, since the paper
    prints contours, not values)."""
    wl = W.lax_liu_2d(config)
    with F.Solver.from_workload(wl) as s:
        s.init_riemann(wl.states, wl.xsplit, wl.ysplit)
        s.step(wl.nsteps)
        n, _, _, T = s.moments()
    lo, hi = rho_range
    print(f"C{config}: rho in [{n.min():.4f}, {n.max():.4f}], paper contours [{lo}, {hi}]")
    assert np.isfinite(n).all() and (T > 0).all()
    assert abs(n.min() - lo) < 0.015 and abs(n.max() - hi) < 0.015 * hi
