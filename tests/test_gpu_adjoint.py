"""The discrete adjoint of the IMEX step (1-D, binary64), called through the
C ABI and through the torch.autograd.Function of the binding.

What fixes the adjoint:
* the transpose (dot-product) identity <Gbar, J dF> = <J^T Gbar, dF>, with
  J dF taken by central differences of the forward step (the limiter's
  selections do not change within +-h on smooth data, so J is the Jacobian
  the adjoint transposes);
* central finite differences (h = 1e-6 relative, binary64) of the loss with
  respect to every parameter: the six blended (rho, u, P), gamma and tau;
* the same derivatives taken by central differences of the CPU oracle (the
  binary64 reference gradient), which shares no code with the CUDA path;
* checkpoint spacing: the adjoint of the state is the same array whatever
  the number of steps between checkpoints.

Tolerances.  A central difference with step h carries a truncation error of
order h^2 times the third derivative and a rounding error of order
eps |S| / (h |dS/dp|).  For the fields and gamma, h = 1e-6 (relative) gives
errors measured below 1e-7; the bound is 1e-6.  tau acts only through the
non-equilibrium parts of the stages (of order tau), so a relative step of
1e-6 moves each population by about 1e5 ulps per step and the difference
quotient is noise-limited: measured against the adjoint, 2.8e-4 at h = 1e-6,
3.6e-5 at 1e-5, 7e-6 at 1e-4 and 5e-7 at 1e-3.  The tau derivatives are
therefore checked with h = 1e-3 (relative; truncation about 1e-7) and a
bound of 2e-5.
"""
import math

import numpy as np
import pytest

from paper_1909_08390_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1909_08390_gb300 import build as B, fdlb
    B.build()
    fdlb.load()
    return fdlb


@pytest.fixture(scope="module")
def torch():
    import torch as T
    return T


def make_ctx(F, nx, Q=(8, 8), gamma=1.4, tau=1e-5, dt=2e-5, precision=None, d=1, bc=None):
    g = F.fdlb_grid(d, nx, nx if d == 2 else 1, -0.5, 0.5, -0.5, 0.5,
                    F.FDLB_BC_OUTLET if bc is None else bc)
    return F.fdlb_create(g, Q[0], Q[1], gamma, tau, dt, None,
                         F.FDLB_FP64 if precision is None else precision, None)


def smooth_state(F, torch, ctx, nx, seed=3, noneq=0.02):
    """Equilibrium of smooth fields times (1 + noneq * smooth noise): a valid
    state away from equilibrium, so the relaxation terms are exercised."""
    n, u, T = W.smooth_fields_1d(nx, seed=seed, amp=0.1)
    dev = "cuda"
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev).contiguous()
    F.fdlb_init_fields(ctx, t(n), t(u), t(T))
    P = F.fdlb_npop(ctx)
    S = torch.empty((P, nx), dtype=torch.float64, device=dev)
    F.fdlb_get_state(ctx, S, True)
    noise = t(W.smooth_random_populations((P, nx), seed=seed + 1, amp=1.0) - 1.0)
    return (S * (1.0 + noneq * noise)).contiguous()


def run_state(F, torch, ctx, S0, nsteps):
    F.fdlb_set_state(ctx, S0.contiguous(), True)
    F.fdlb_step(ctx, nsteps)
    out = torch.empty_like(S0)
    F.fdlb_get_state(ctx, out, True)
    torch.cuda.synchronize()
    return out


def adjoint_of(F, torch, ctx, S0, nsteps, every, Gbar):
    F.fdlb_set_state(ctx, S0.contiguous(), True)
    ck = torch.empty((nsteps // every + 1,) + tuple(S0.shape), dtype=torch.float64, device="cuda")
    F.fdlb_forward_ckpt(ctx, nsteps, every, ck)
    Fb = Gbar.clone().contiguous()
    dg, dtau = F.fdlb_adjoint(ctx, nsteps, every, ck, Fb)
    torch.cuda.synchronize()
    return Fb, dg, dtau, ck


@pytest.mark.parametrize("Q,nx,nsteps", [((8, 8), 300, 1), ((5, 3), 173, 1), ((3, 3), 97, 1),
                                         ((8, 8), 300, 12)])
def test_dot_product_state(F, torch, Q, nx, nsteps):
    """<Gbar, J dF> (central differences of the forward) = <J^T Gbar, dF>."""
    ctx = make_ctx(F, nx, Q)
    try:
        S0 = smooth_state(F, torch, ctx, nx)
        P = S0.shape[0]
        g = torch.Generator(device="cpu").manual_seed(11)
        Gbar = torch.randn((P, nx), generator=g, dtype=torch.float64).cuda()
        dF = torch.as_tensor(W.smooth_random_populations((P, nx), seed=5, amp=1.0) - 1.0,
                             device="cuda") * S0
        h = 1e-6
        Sp = run_state(F, torch, ctx, S0 + h * dF, nsteps)
        Sm = run_state(F, torch, ctx, S0 - h * dF, nsteps)
        lhs = float((Gbar * (Sp - Sm)).sum()) / (2 * h)
        Fb, _, _, _ = adjoint_of(F, torch, ctx, S0, nsteps, 5, Gbar)
        rhs = float((Fb * dF).sum())
        err = abs(lhs - rhs) / abs(rhs)
        print(f"dot product Q={Q} nx={nx} steps={nsteps}: rel err {err:.3e}")
        assert err < (1e-7 if nsteps == 1 else 1e-6), (lhs, rhs, err)
    finally:
        F.fdlb_destroy(ctx)


@pytest.mark.parametrize("d,Q,nx", [(1, (8, 8), 300), (1, (5, 3), 77), (2, (8, 8), 37),
                                    (2, (5, 3), 29)])
def test_moments_adjoint_dot_product(F, torch, d, Q, nx):
    """fdlb_moments_adjoint is the transpose of the moment map (n, u, T)(F) of
    Eq. (Moments_discrete): <mbar, J dF> by central differences of
    fdlb_moments equals <J^T mbar, dF>; with nbar alone it is nbar on every
    phi population and 0 on every chi population (n = sum phi)."""
    ctx = make_ctx(F, nx, Q, d=d)
    try:
        P = F.fdlb_npop(ctx)
        shape = (P, nx) if d == 1 else (P, nx, nx)
        S0 = torch.as_tensor(W.smooth_random_populations(shape, seed=9, amp=0.2), device="cuda")
        dF = torch.as_tensor(W.smooth_random_populations(shape, seed=10, amp=1.0) - 1.0,
                             device="cuda") * S0
        g = torch.Generator(device="cpu").manual_seed(3)
        cells = shape[1:]
        mbar = [torch.randn(cells, generator=g, dtype=torch.float64).cuda() for _ in range(4)]
        if d == 1:
            mbar[2] = None

        def moments(S):
            F.fdlb_set_state(ctx, S.contiguous(), True)
            out = [torch.empty(cells, dtype=torch.float64, device="cuda") for _ in range(4)]
            F.fdlb_moments(ctx, out[0], out[1], out[2] if d == 2 else None, out[3], True)
            torch.cuda.synchronize()
            return out

        h = 1e-6
        mp, mm = moments(S0 + h * dF), moments(S0 - h * dF)
        lhs = sum(float((b * (x - y)).sum()) for b, x, y in zip(mbar, mp, mm) if b is not None)
        lhs /= 2 * h
        F.fdlb_set_state(ctx, S0.contiguous(), True)
        Fb = torch.empty(shape, dtype=torch.float64, device="cuda")
        F.fdlb_moments_adjoint(ctx, *mbar, Fb)
        rhs = float((Fb * dF).sum())
        assert abs(lhs - rhs) <= 1e-8 * abs(rhs), (lhs, rhs)
        F.fdlb_moments_adjoint(ctx, mbar[0], None, None, None, Fb)
        nphi = Q[0] ** d
        torch.testing.assert_close(Fb[:nphi], mbar[0].expand_as(Fb[:nphi]), rtol=0, atol=0)
        assert float(Fb[nphi:].abs().max()) == 0.0
    finally:
        F.fdlb_destroy(ctx)


@pytest.mark.parametrize("which", ["gamma", "tau"])
def test_parameter_derivatives_of_steps(F, torch, which):
    """dparams of fdlb_adjoint against central differences of the steps in
    gamma (D + K = 2/(gamma - 1)) and tau (lambda = dt/tau)."""
    nx, nsteps, gamma, tau = 256, 10, 1.4, 1e-5
    ctx = make_ctx(F, nx, gamma=gamma, tau=tau)
    try:
        S0 = smooth_state(F, torch, ctx, nx, noneq=0.05)
        g = torch.Generator(device="cpu").manual_seed(12)
        Gbar = torch.randn(tuple(S0.shape), generator=g, dtype=torch.float64).cuda()
        _, dg, dtau, _ = adjoint_of(F, torch, ctx, S0, nsteps, 4, Gbar)
    finally:
        F.fdlb_destroy(ctx)
    base = gamma if which == "gamma" else tau
    h = (1e-6 if which == "gamma" else 1e-3) * base
    vals = []
    for sgn in (1, -1):
        kw = {"gamma": gamma, "tau": tau}
        kw[which] = base + sgn * h
        c = make_ctx(F, nx, **kw)
        try:
            vals.append(run_state(F, torch, c, S0, nsteps))
        finally:
            F.fdlb_destroy(c)
    fd = float((Gbar * (vals[0] - vals[1])).sum()) / (2 * h)
    got = dg if which == "gamma" else dtau
    print(f"d/d{which}: adjoint {got:.12e} fd {fd:.12e} rel {abs(got - fd) / abs(fd):.3e}")
    assert abs(got - fd) <= (1e-6 if which == "gamma" else 2e-5) * abs(fd), (which, got, fd)


def test_checkpoint_spacing_invariance(F, torch):
    """Fbar and the gamma and tau adjoints are bitwise the same for every
    checkpoint spacing: each segment's recomputation is bitwise the forward
    run, and the scalar adjoints are summed without atomics, per block in
    warp order and over blocks in block order.  A second run with the same
    spacing gives the same bits too.  Covers a ragged last segment."""
    nx, nsteps = 200, 23
    ctx = make_ctx(F, nx)
    try:
        S0 = smooth_state(F, torch, ctx, nx)
        g = torch.Generator(device="cpu").manual_seed(13)
        Gbar = torch.randn(tuple(S0.shape), generator=g, dtype=torch.float64).cuda()
        ref = None
        for every in (1, 5, 23, 50):
            Fb, dg, dtau, ck = adjoint_of(F, torch, ctx, S0, nsteps, every, Gbar)
            if ref is None:
                ref = (Fb, dg, dtau)
                # the checkpointed forward is the plain run: its checkpoints
                # are the states after 0, 1, ..., nsteps steps
                assert torch.equal(ck[0], S0)
                assert torch.equal(ck[nsteps], run_state(F, torch, ctx, S0, nsteps))
                continue
            assert torch.equal(Fb, ref[0]), every
            assert dg == ref[1] and dtau == ref[2], (every, dg - ref[1], dtau - ref[2])
        Fb, dg, dtau, _ = adjoint_of(F, torch, ctx, S0, nsteps, 1, Gbar)
        assert torch.equal(Fb, ref[0]) and dg == ref[1] and dtau == ref[2]
    finally:
        F.fdlb_destroy(ctx)


def test_zero_steps_and_state_kept(F, torch):
    nx = 64
    ctx = make_ctx(F, nx)
    try:
        S0 = smooth_state(F, torch, ctx, nx)
        Gbar = torch.ones_like(S0)
        Fb, dg, dtau, _ = adjoint_of(F, torch, ctx, S0, 0, 50, Gbar)
        assert torch.equal(Fb, Gbar) and dg == 0.0 and dtau == 0.0
        # a reverse pass leaves the context's state (the forward's end state) alone
        F.fdlb_set_state(ctx, S0, True)
        ck = torch.empty((3,) + tuple(S0.shape), dtype=torch.float64, device="cuda")
        F.fdlb_forward_ckpt(ctx, 10, 5, ck)
        end = torch.empty_like(S0)
        F.fdlb_get_state(ctx, end, True)
        F.fdlb_adjoint(ctx, 10, 5, ck, Gbar.clone())
        after = torch.empty_like(S0)
        F.fdlb_get_state(ctx, after, True)
        torch.cuda.synchronize()
        assert torch.equal(end, after)
        # and the next step continues from it as if no reverse pass had run
        F.fdlb_step(ctx, 1)
        nxt = torch.empty_like(S0)
        F.fdlb_get_state(ctx, nxt, True)
        torch.cuda.synchronize()
        assert torch.equal(nxt, run_state(F, torch, ctx, end, 1))
    finally:
        F.fdlb_destroy(ctx)


def test_unsupported_contexts_rejected(F, torch):
    for kw in ({"precision": 1}, {"d": 2}, {"bc": 1}):
        nx = 32
        ctx = make_ctx(F, nx, **kw)
        try:
            z = torch.zeros(2 * F.fdlb_state_bytes(ctx) // 8, dtype=torch.float64, device="cuda")
            with pytest.raises(F.FdlbError) as ei:
                F.fdlb_forward_ckpt(ctx, 1, 1, z)
            assert ei.value.code == F.FDLB_EINVAL
            with pytest.raises(F.FdlbError):
                F.fdlb_adjoint(ctx, 1, 1, z, z)
        finally:
            F.fdlb_destroy(ctx)


def test_init_fields_parity_and_adjoint(F, torch, oracle):
    """fdlb_init_fields against the oracle's equilibrium of the same fields;
    its adjoint by the dot-product identity (the map is smooth)."""
    nx = 150
    for Q in ((8, 8), (5, 3)):
        ctx = make_ctx(F, nx, Q, gamma=1.3)
        try:
            n, u, T = W.smooth_fields_1d(nx, seed=9, amp=0.2)
            t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda").contiguous()
            F.fdlb_init_fields(ctx, t(n), t(u), t(T))
            P = F.fdlb_npop(ctx)
            S = torch.empty((P, nx), dtype=torch.float64, device="cuda")
            F.fdlb_get_state(ctx, S, True)
            pr = oracle.Problem(d=1, nx=nx, Qphi=Q[0], Qchi=Q[1], gamma=1.3, tau=1e-5, dt=2e-5)
            want = oracle.init_fields(pr, n, u, None, T)
            got = S.cpu().numpy()
            assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
            # dot product: d/deps <Fbar, Feq(fields + eps dfields)>
            g = np.random.default_rng(4)
            dn, du, dT = (g.standard_normal(nx) * 0.1 for _ in range(3))
            Fbar = torch.as_tensor(g.standard_normal((P, nx)), device="cuda").contiguous()
            nb, ub, Tb = (torch.empty(nx, dtype=torch.float64, device="cuda") for _ in range(3))
            dk = F.fdlb_init_fields_adjoint(ctx, Fbar, t(n), t(u), t(T), nb, ub, Tb)
            rhs = float((nb.cpu().numpy() * dn + ub.cpu().numpy() * du + Tb.cpu().numpy() * dT).sum())
            h = 1e-6
            Fp = oracle.init_fields(pr, n + h * dn, u + h * du, None, T + h * dT)
            Fm = oracle.init_fields(pr, n - h * dn, u - h * du, None, T - h * dT)
            lhs = float((Fbar.cpu().numpy() * (Fp - Fm)).sum()) / (2 * h)
            assert abs(lhs - rhs) <= 1e-7 * abs(rhs), (lhs, rhs)
            # gamma: chi^eq = (D + K - 1) T phi-shape, D + K = 2/(gamma - 1)
            hg = 1e-6
            pp = oracle.Problem(d=1, nx=nx, Qphi=Q[0], Qchi=Q[1], gamma=1.3 + hg, tau=1e-5, dt=2e-5)
            pm = oracle.Problem(d=1, nx=nx, Qphi=Q[0], Qchi=Q[1], gamma=1.3 - hg, tau=1e-5, dt=2e-5)
            fdg = float((Fbar.cpu().numpy() * (oracle.init_fields(pp, n, u, None, T)
                                               - oracle.init_fields(pm, n, u, None, T))).sum()) / (2 * hg)
            assert abs(dk - fdg) <= 1e-7 * abs(fdg), (dk, fdg)
        finally:
            F.fdlb_destroy(ctx)


# ---- end to end: loss of the final density, torch.autograd ---------------------

def gpu_loss(F, torch, run, prm, gamma, tau, target, grad):
    dx = (run.x1 - run.x0) / run.nx
    n0, u0, T0 = F.blended_fields(prm, run.nx, run.x0, run.x1, run.width)
    if grad:
        n = F.density_run(n0, u0, T0, gamma, tau, run.spec())
    else:
        n = F.density_forward(n0, u0, T0, gamma, tau, run.spec())
    return dx * ((n - target) ** 2).sum()


def autograd_gradient(F, torch, run, target):
    prm = torch.as_tensor(run.params(), device="cuda").requires_grad_(True)
    gamma = torch.tensor(run.gamma, dtype=torch.float64, device="cuda", requires_grad=True)
    tau = torch.tensor(run.tau, dtype=torch.float64, device="cuda", requires_grad=True)
    L = gpu_loss(F, torch, run, prm, gamma, tau, target, True)
    L.backward()
    return float(L.detach()), np.concatenate([prm.grad.cpu().numpy(),
                                              [float(gamma.grad), float(tau.grad)]])


HREL = np.array([1e-6] * 7 + [1e-3])  # relative steps: six states, gamma, tau
TOL = np.array([1e-6] * 7 + [2e-5])


def fd_gradient(loss_of, run):
    """Central differences in the 8 parameters (h = HREL * max(|p|, 1) for
    the six states, HREL * p for gamma and tau)."""
    base = np.concatenate([run.params(), [run.gamma, run.tau]])
    out = np.zeros(8)
    for i in range(8):
        h = HREL[i] * (max(abs(base[i]), 1.0) if i < 6 else base[i])
        p, m = base.copy(), base.copy()
        p[i] += h
        m[i] -= h
        out[i] = (loss_of(p) - loss_of(m)) / (2 * h)
    return out


def check_gradient(got, want, tol, floor):
    """Per component, relative to max(|want_i|, floor * max|want|)."""
    scale = np.maximum(np.abs(want), floor * np.abs(want).max())
    err = np.abs(got - want) / scale
    print("gradient rel err per parameter:", np.array2string(err, precision=3))
    assert (err < tol).all(), (got, want, err)
    return err.max()


def test_autograd_against_fd_and_oracle(F, torch, oracle):
    """Small run (256 cells, 120 steps, checkpoints every 50): the autograd
    gradient against central differences of the GPU forward and of the
    CPU oracle (the binary64 reference gradient)."""
    run = W.adjoint_1d(nx=256, nsteps=120, every=50)
    target_np = W.smooth_target(run.nx, run.x0, run.x1, run.target_seed)
    target = torch.as_tensor(target_np, device="cuda")
    L, g = autograd_gradient(F, torch, run, target)

    def gpu_loss_of(v):
        prm = torch.as_tensor(v[:6], device="cuda")
        return float(gpu_loss(F, torch, run, prm, v[6], v[7], target, False))

    assert abs(gpu_loss_of(np.concatenate([run.params(), [run.gamma, run.tau]])) - L) == 0.0
    fd = fd_gradient(gpu_loss_of, run)
    check_gradient(g, fd, TOL, 1e-3)

    dx = (run.x1 - run.x0) / run.nx
    x = W.cell_centres(run.nx, run.x0, run.x1)

    def oracle_loss_of(v):
        pr = oracle.Problem(d=1, nx=run.nx, x0=run.x0, x1=run.x1, Qphi=run.Q, Qchi=run.Q,
                            gamma=v[6], tau=v[7], dt=run.dt)
        rho, u, P = W.blend_states(v[:6], x, run.width, np.tanh)
        S = oracle.step(pr, oracle.init_fields(pr, rho, u, None, P / rho), run.nsteps)
        n = oracle.moments(pr, S)[0]
        return dx * float(((n - target_np) ** 2).sum())

    ref = fd_gradient(oracle_loss_of, run)
    check_gradient(g, ref, TOL, 1e-3)


def test_adjoint_sod_blend_2048_cells_2000_steps(F, torch):
    """The full differentiable run: 2048 cells, Q = 8, gamma = 7/5,
    tau = 1e-5, dt = 2e-5, 2000 steps, checkpoints every 50 steps."""
    run = W.adjoint_1d()
    target = torch.as_tensor(W.smooth_target(run.nx, run.x0, run.x1, run.target_seed),
                             device="cuda")
    L, g = autograd_gradient(F, torch, run, target)
    assert math.isfinite(L) and np.isfinite(g).all()

    def gpu_loss_of(v):
        prm = torch.as_tensor(v[:6], device="cuda")
        return float(gpu_loss(F, torch, run, prm, v[6], v[7], target, False))

    fd = fd_gradient(gpu_loss_of, run)
    check_gradient(g, fd, TOL, 1e-3)
