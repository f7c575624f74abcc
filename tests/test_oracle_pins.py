"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden/paper_values.json), textbook values of the exact
Sod solution, hand-worked MP-9 examples, library routines (numpy's
Gauss-Hermite rule, scipy quadrature), closed forms (Gaussian moments, the
linear stability functions of the Butcher tableaux) and invariants
(conservation, symmetry, monotonicity preservation, order of accuracy).
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1909_08390_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Sec. II: Gauss-Hermite quadrature
# --------------------------------------------------------------------------

@pytest.mark.parametrize("Q", [1, 2, 3, 4, 5, 6, 8, 10, 12])
def test_gauss_hermite_matches_numpy(oracle, Q):
    p, w = oracle.gauss_hermite(Q)
    pn, wn = np.polynomial.hermite_e.hermegauss(Q)
    np.testing.assert_allclose(p, pn, rtol=0, atol=1e-13)
    np.testing.assert_allclose(w, wn / math.sqrt(2 * math.pi), rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("Q", [3, 5, 8])
def test_gauss_hermite_moments_exact(oracle, Q):
    # sum_k w_k p_k^m = E[Z^m], Z ~ N(0,1): (m-1)!! for even m, 0 for odd, m <= 2Q-1
    p, w = oracle.gauss_hermite(Q)
    for m in range(0, 2 * Q):
        exact = 0.0 if m % 2 else float(np.prod(np.arange(m - 1, 0, -2))) if m > 0 else 1.0
        got = float(np.sum(w * p ** m))
        assert abs(got - exact) <= 1e-12 * max(1.0, exact), (Q, m, got, exact)


def test_gauss_hermite_q8_roots_printed(oracle):
    # roots of He_8 to six digits
    p, _ = oracle.gauss_hermite(8)
    np.testing.assert_allclose(p[4:], [0.539080, 1.636519, 2.802486, 4.144547], atol=1e-6)
    np.testing.assert_allclose(p[:4], -p[4:][::-1], atol=1e-14)


# --------------------------------------------------------------------------
# Sec. II, Eq. (gExpanded): equilibria
# --------------------------------------------------------------------------

@pytest.mark.parametrize("Q", [3, 5, 8])
@pytest.mark.parametrize("u,T", [(0.0, 1.0), (0.3, 0.7), (-0.8, 1.4), (1.1, 0.2)])
def test_equilibrium_factor_is_gaussian_projection(oracle, Q, u, T):
    """g_k = w_k sum_l He_l(p_k)/l! * a_l with a_l = int He_l(p) N(p; u, T) dp,
    the coefficients computed here by numerical integration (scipy) and He by
    numpy's hermeval: the truncated Hermite expansion of the Maxwellian."""
    import warnings

    from scipy.integrate import IntegrationWarning, quad
    p, w = oracle.gauss_hermite(Q)
    a = []
    for l in range(Q):
        c = np.zeros(l + 1)
        c[l] = 1.0
        f = lambda x: np.polynomial.hermite_e.hermeval(x, c) * math.exp(-(x - u) ** 2 / (2 * T)) / math.sqrt(2 * math.pi * T)
        # the tolerances ask for more than binary64 round-off allows on the
        # higher orders; quad then warns, and the comparison below (1e-10)
        # judges the result
        with warnings.catch_warnings():
            warnings.simplefilter("ignore", IntegrationWarning)
            a.append(quad(f, u - 40 * math.sqrt(T), u + 40 * math.sqrt(T), epsabs=1e-14,
                          epsrel=1e-14, limit=200)[0])
    expect = np.zeros(Q)
    for l in range(Q):
        c = np.zeros(l + 1)
        c[l] = 1.0
        expect += np.polynomial.hermite_e.hermeval(p, c) / math.factorial(l) * a[l]
    expect *= w
    got = oracle.g_axis(Q, u, T)
    np.testing.assert_allclose(got, expect, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("Q", [3, 5, 8])
def test_equilibrium_factor_gaussian_moments(oracle, Q):
    # sum_k g_k p_k^m = E[X^m], X ~ N(u, T), for m <= Q-1 (Sec. II: exact recovery
    # of the moments up to order Q-1 per axis)
    from scipy.stats import norm
    p, _ = oracle.gauss_hermite(Q)
    for (u, T) in [(0.2, 0.9), (-0.7, 0.3), (1.0, 1.7)]:
        g = oracle.g_axis(Q, u, T)
        for m in range(Q):
            exact = norm(loc=u, scale=math.sqrt(T)).moment(m)
            assert abs(np.sum(g * p ** m) - exact) < 1e-11 * max(1, abs(exact)), (u, T, m)


@pytest.mark.parametrize("d,Qphi,Qchi", [(1, 8, 8), (1, 5, 3), (2, 8, 8), (2, 5, 3), (1, 3, 1)])
def test_equilibrium_reproduces_moments(oracle, d, Qphi, Qchi):
    rng = np.random.default_rng(1)
    pr = oracle.Problem(d=d, nx=1, ny=1, Qphi=Qphi, Qchi=Qchi, gamma=float(rng.uniform(1.1, 1.6)))
    for _ in range(5):
        n = rng.uniform(0.1, 2.0)
        u = rng.uniform(-1, 1, size=d)
        T = rng.uniform(0.2, 2.0)
        feq = oracle.equilibrium(pr, n, u, T)
        shape = (pr.npop, 1, 1) if d == 2 else (pr.npop, 1)
        nn, ux, uy, TT = oracle.moments(pr, feq.reshape(shape))
        assert abs(nn.item() - n) < 1e-14 * n
        assert abs(ux.item() - u[0]) < 1e-13
        if d == 2:
            assert abs(uy.item() - u[1]) < 1e-13
        assert abs(TT.item() - T) < 1e-13 * max(1, T)


def test_population_counts_printed(oracle):
    g = golden("paper_values.json")
    assert oracle.Problem(d=1, Qphi=5, Qchi=3).npop == g["sod"]["populations"]
    assert oracle.Problem(d=2, Qphi=5, Qchi=3).npop == g["riemann_2d"]["populations"]


# --------------------------------------------------------------------------
# Table I: the IMEX-SSP3(4,3,3) tableaux
# --------------------------------------------------------------------------

def _tab(oracle):
    t = oracle.paper_tableau()
    return (np.array(t["At"]), np.array(t["A"]), np.array(t["wt"]), np.array(t["w"]))


def test_tableau_printed_constants(oracle):
    g = golden("paper_values.json")["tableau"]
    At, A, wt, w = _tab(oracle)
    al, be, et = g["alpha"], g["beta"], g["eta"]
    np.testing.assert_array_equal(At, np.array(g["At"], dtype=float))
    np.testing.assert_allclose(wt, g["wt"], rtol=0, atol=1e-16)
    np.testing.assert_allclose(w, g["w"], rtol=0, atol=1e-16)
    np.testing.assert_allclose(np.diag(A), [al] * 4, rtol=0, atol=0)
    assert A[1, 0] == -al and A[2, 1] == 1 - al and A[3, 0] == be and A[3, 1] == et
    assert abs(A[3, 2] - (0.5 - be - et - al)) < 1e-17
    np.testing.assert_allclose(At.sum(1), g["c_explicit"], atol=1e-16)
    np.testing.assert_allclose(A.sum(1), [al, 0.0, 1.0, 0.5], atol=1e-15)


def test_tableau_order_three_conditions(oracle):
    """Order conditions of additive (IMEX) Runge-Kutta methods up to order 3,
    explicit, implicit and coupling; they pin all tableau entries."""
    At, A, wt, w = _tab(oracle)
    ct, c = At.sum(1), A.sum(1)
    conds = [
        wt.sum() - 1, w.sum() - 1,
        wt @ ct - .5, w @ c - .5, wt @ c - .5, w @ ct - .5,
        wt @ ct ** 2 - 1 / 3, w @ c ** 2 - 1 / 3, wt @ (ct * c) - 1 / 3, wt @ (c * c) - 1 / 3,
        w @ (ct * ct) - 1 / 3, w @ (ct * c) - 1 / 3,
        wt @ At @ ct - 1 / 6, w @ A @ c - 1 / 6, wt @ At @ c - 1 / 6, wt @ A @ ct - 1 / 6,
        wt @ A @ c - 1 / 6, w @ At @ ct - 1 / 6, w @ At @ c - 1 / 6, w @ A @ ct - 1 / 6,
    ]
    assert max(abs(x) for x in conds) < 1e-13


def _stability(Amat, b, z):
    r = Amat.shape[0]
    return 1 + z * b @ np.linalg.solve(np.eye(r) - z * Amat, np.ones(r))


@pytest.mark.parametrize("lam", [0.01, 0.5, 3.0, 50.0, 1e4])
def test_pure_relaxation_follows_implicit_stability_function(oracle, lam):
    """Spatially uniform non-equilibrium data (periodic): no advection, so each
    population obeys dF/dt = -(F - F_eq)/tau with F_eq fixed by the conserved
    moments; one step multiplies F - F_eq by R(z) = 1 + z w^T (I - zA)^{-1} 1,
    z = -dt/tau (numpy linear algebra on the tableau)."""
    pr = oracle.Problem(d=1, nx=12, bc=1, Qphi=8, Qchi=8, gamma=1.4, tau=1.0, dt=lam)
    rng = np.random.default_rng(3)
    feq = oracle.equilibrium(pr, 0.9, [0.3], 1.2)
    pert = rng.uniform(-0.05, 0.05, size=pr.npop) * feq.max()
    F0 = np.repeat((feq + pert)[:, None], pr.nx, axis=1)
    # the equilibrium of F0's own moments
    n, u, _, T = oracle.moments(pr, F0)
    feq0 = oracle.equilibrium(pr, n[0], [u[0]], T[0])
    F1 = oracle.step(pr, F0, 1)
    _, A, _, w = _tab(oracle)
    R = _stability(A, w, -lam)
    expect = feq0[:, None] + R * (F0 - feq0[:, None])
    np.testing.assert_allclose(F1, expect, rtol=0, atol=1e-14 * np.abs(F0).max() * max(1, lam))


# Shu-Osher SSP-RK3 on the whole right-hand side as a 4-stage tableau (stages
# F^n, F^n, F^n + dt f(F^n), F^n + dt (f(F^n) + f(F^(3)))/4): the fully
# explicit comparator of Sec. VI's dt/tau claim
SSPRK3 = {"At": [[0, 0, 0, 0], [0, 0, 0, 0], [0, 1, 0, 0], [0, 0.25, 0.25, 0]],
          "A": [[0, 0, 0, 0], [0, 0, 0, 0], [0, 1, 0, 0], [0, 0.25, 0.25, 0]],
          "wt": [0, 1 / 6, 1 / 6, 2 / 3], "w": [0, 1 / 6, 1 / 6, 2 / 3]}


@pytest.mark.parametrize("lam", [0.5, 1.0, 2.0, 2.5, 3.0])
def test_explicit_comparator_relaxation_is_taylor_polynomial(oracle, lam):
    """With the explicit tableau, spatially uniform non-equilibrium data relax
    by the cubic Taylor polynomial of exp(z), z = -dt/tau, per step: stable
    (|R| <= 1) for dt/tau up to about 2.51 and growing beyond."""
    pr = oracle.Problem(d=1, nx=8, bc=1, Qphi=8, Qchi=8, gamma=1.4, tau=1.0, dt=lam,
                        tableau=SSPRK3)
    rng = np.random.default_rng(4)
    feq = oracle.equilibrium(pr, 1.1, [-0.2], 0.9)
    pert = rng.uniform(-0.05, 0.05, size=pr.npop) * feq.max()
    F0 = np.repeat((feq + pert)[:, None], pr.nx, axis=1)
    n, u, _, T = oracle.moments(pr, F0)
    feq0 = oracle.equilibrium(pr, n[0], [u[0]], T[0])
    F1 = oracle.step(pr, F0, 1)
    z = -lam
    R = 1 + z + z * z / 2 + z ** 3 / 6
    np.testing.assert_allclose(F1, feq0[:, None] + R * (F0 - feq0[:, None]), rtol=0,
                               atol=1e-14 * np.abs(F0).max() * max(1, lam ** 3))
    assert (abs(R) <= 1.0) == (lam <= 2.5)


@pytest.mark.parametrize("p_sign", [1, -1])
@pytest.mark.parametrize("theta_cells", [32, 64])
def test_linear_advection_follows_explicit_stability_function(oracle, p_sign, theta_cells):
    """No collisions (tau <= 0).  A smooth periodic mode per population with the
    limiter leaving F^L unchanged: the scheme is linear, each Fourier mode is
    an eigenvector of the flux-difference operator with eigenvalue
    (p/ds) sigma(theta)(1 - e^{-i theta}) (p > 0; mirrored for p < 0), and one
    step multiplies it by the explicit stability function of (At, wt)."""
    nx = 128
    pr = oracle.Problem(d=1, nx=nx, bc=1, Qphi=3, Qchi=1, gamma=1.4, tau=-1.0, dt=2e-3,
                        x0=0.0, x1=1.0)
    ds = 1.0 / nx
    theta = 2 * math.pi / theta_cells
    s = np.arange(nx)
    c = np.array(golden("paper_values.json")["mp9"]["coefficients_over_2520"]) / 2520.0
    p, _ = oracle.gauss_hermite(3)
    At, _, wt, _ = _tab(oracle)
    # one velocity of the requested sign, others at rest (zero momentum node)
    F0 = np.ones((pr.npop, nx))
    k = 2 if p_sign > 0 else 0
    F0[k] = 1.0 + 0.01 * np.cos(theta * s)
    F1 = oracle.step(pr, F0, 1)
    pk = p[k]
    th = theta if pk > 0 else -theta  # mirrored line sees the mode with opposite phase speed
    sigma = np.sum(c * np.exp(1j * th * np.arange(-4, 5)))
    eig = abs(pk) / ds * sigma * (1 - np.exp(-1j * th))
    R = _stability(At, wt, -pr.dt * eig)
    expect = 1.0 + 0.01 * np.real(R * np.exp(1j * theta * s))
    np.testing.assert_allclose(F1[k], expect, rtol=0, atol=1e-14)
    np.testing.assert_allclose(F1[1], 1.0, rtol=0, atol=1e-15)  # p = 0 node does not move


# --------------------------------------------------------------------------
# Sec. IV: MP-9 advection
# --------------------------------------------------------------------------

def test_mp9_hand_worked_examples(oracle):
    for e in golden("mp9_hand_examples.json")["examples"]:
        val, lim = oracle.mp9_face(e["v"])
        assert lim == e["limited"], e
        assert abs(val - e["face"]) < 1e-15, (e, val)


def test_mp9_coefficients_printed_sum_to_one(oracle):
    c = golden("paper_values.json")["mp9"]["coefficients_over_2520"]
    assert sum(c) == 2520
    # F^L of a constant is that constant
    val, lim = oracle.mp9_face([3.25] * 9)
    assert val == 3.25 and not lim


@pytest.mark.parametrize("deg", range(0, 9))
def test_mp9_exact_on_polynomial_cell_averages(oracle, deg):
    """For cell averages of a polynomial of degree <= 8, the 9-point interface
    value equals the point value at the interface (limiter inactive on
    monotone data)."""
    rng = np.random.default_rng(deg)
    # monotone increasing polynomial on the stencil: integral of a positive one
    for trial in range(3):
        roots = rng.uniform(-10, -6, size=max(deg - 1, 0))
        dP = np.poly1d(np.poly(roots)) if deg >= 1 else np.poly1d([0.0])
        P = np.polyint(dP) if deg >= 1 else np.poly1d([rng.uniform(-1, 1)])
        P = P + rng.uniform(-1, 1)
        if deg == 0:
            P = np.poly1d([rng.uniform(-1, 1)])
        h = 0.1
        Pint = np.polyint(P)
        edges = (np.arange(-4, 6) - 0.5) * h  # cell j in [(j-1/2)h, (j+1/2)h]
        avg = (Pint(edges[1:]) - Pint(edges[:-1])) / h
        val, lim = oracle.mp9_face(avg)
        exact = P(0.5 * h)
        if deg > 0:
            assert not lim
        assert abs(val - exact) < 1e-10 * max(1, abs(exact)), (deg, val, exact)


def test_mp9_translation_and_scaling_equivariance(oracle):
    """Every operation of the limiter is translation-equivariant and positively
    homogeneous: face(a v + b) = a face(v) + b for a > 0, and odd: face(-v) = -face(v)."""
    rng = np.random.default_rng(7)
    for _ in range(300):
        v = rng.normal(size=9) * rng.choice([0.01, 1, 100])
        if rng.uniform() < 0.5:
            v = np.cumsum(np.abs(v))  # monotone
        a, b = rng.uniform(0.25, 4), rng.uniform(-5, 5)
        f0, l0 = oracle.mp9_face(v)
        f1, l1 = oracle.mp9_face(a * v + b)
        f2, l2 = oracle.mp9_face(-v)
        scale = np.abs(v).max() * a + abs(b)
        assert abs(f1 - (a * f0 + b)) < 1e-12 * scale
        assert abs(f2 + f0) < 1e-12 * np.abs(v).max()


def test_mp9_monotonicity_preservation(oracle):
    """Suresh & Huynh's MP constraint: with alpha = 4, one forward-Euler step of
    the flux-difference form at CFL <= 1/(1+alpha) maps monotone data to
    monotone data with no new extrema.  Checked on random monotone profiles
    with jumps, for both signs of the velocity."""
    rng = np.random.default_rng(11)
    cfl = 1.0 / 5.0
    for trial in range(40):
        n = 60
        inc = np.abs(rng.normal(size=n)) * (rng.uniform(size=n) < 0.3)
        inc[n // 2] += rng.uniform(1, 5)
        F = 1.0 + np.cumsum(inc)
        if trial % 2:
            F = F[::-1].copy()
        for p in (1.0, -1.0):
            ds = 0.01
            dt = cfl * ds / abs(p)
            LF = oracle.advect_line(F, p, ds, bc=0)
            G = F - dt * LF
            dG = np.diff(G)
            if F[-1] >= F[0]:
                assert dG.min() >= -1e-12, (trial, p, dG.min())
            else:
                assert dG.max() <= 1e-12, (trial, p, dG.max())
            assert G.min() >= F.min() - 1e-12 and G.max() <= F.max() + 1e-12


def test_advection_mirror_symmetry(oracle):
    # p < 0 on a line equals p > 0 on the reversed line, reversed
    rng = np.random.default_rng(5)
    F = rng.uniform(0.1, 2.0, size=50)
    for bc in (0, 1):
        a = oracle.advect_line(F, -1.7, 0.02, bc=bc)
        b = oracle.advect_line(F[::-1].copy(), 1.7, 0.02, bc=bc)[::-1]
        np.testing.assert_array_equal(a, b)


def test_advection_derivative_of_polynomial(oracle):
    """Away from the ghosts, on cell averages of a degree-8 polynomial that is
    monotone on the line, (p dF/dx)_s is p times the cell average of P'."""
    nx, h = 40, 0.05
    P = np.polyint(np.poly1d(np.poly(np.linspace(-9, -6, 7)))) * 1e-6
    Pint = np.polyint(P)
    edges = np.arange(nx + 1) * h
    avg = (Pint(edges[1:]) - Pint(edges[:-1])) / h
    for p in (1.3, -0.7):
        LF = oracle.advect_line(avg, p, h, bc=0)
        exact = p * (P(edges[1:]) - P(edges[:-1])) / h
        sl = slice(6, nx - 6)
        np.testing.assert_allclose(LF[sl], exact[sl], rtol=1e-9, atol=1e-12)


# A non-square 2-D box whose cells are not square: dx = 1.5/24 = 0.0625 and
# dy = 1.0/40 = 0.025, so any mix-up of the two spacings (or of nx and ny)
# changes every y-line's flux difference by a factor of 2.5.
BOX = dict(nx=24, ny=40, x0=0.0, x1=1.5, y0=0.0, y1=1.0)


def test_advect_2d_y_lines_use_dy(oracle):
    """Sec. IV applies the 1-D scheme along each axis with that axis's own
    spacing.  On the box above, a field that varies only along y has no
    x-flux (constant lines give F_hat = F_s exactly), and every population's
    2-D operator equals its 1-D y-line operator with ds = dy, for positive,
    zero and negative p_y.  The y profile is the cell averages of a monotone
    degree-8 polynomial, so away from the ghosts the result is also p_y
    times the polynomial's exact difference quotient over dy."""
    pr = oracle.Problem(d=2, bc=0, Qphi=5, Qchi=3, gamma=1.4, tau=1e-5, dt=1e-3, **BOX)
    nx, ny = BOX["nx"], BOX["ny"]
    dy = (BOX["y1"] - BOX["y0"]) / ny
    P = np.polyint(np.poly1d(np.poly(np.linspace(-9, -6, 7)))) * 1e-6 + 0.5
    Pint = np.polyint(P)
    edges = BOX["y0"] + np.arange(ny + 1) * dy
    col = (Pint(edges[1:]) - Pint(edges[:-1])) / dy
    F = np.empty(pr.shape)
    for k in range(pr.npop):
        F[k] = (1.0 + 0.1 * k) * col[:, None]
    LF = oracle.advect(pr, F)
    p5, _ = oracle.gauss_hermite(5)
    p3, _ = oracle.gauss_hermite(3)
    py = [p5[k // 5] for k in range(25)] + [p3[q // 3] for q in range(9)]
    assert min(py) < 0 < max(py) and 0.0 in py
    sl = slice(6, ny - 6)
    for k in range(pr.npop):
        line = oracle.advect_line(F[k][:, 0].copy(), py[k], dy, bc=0)
        np.testing.assert_array_equal(LF[k], np.repeat(line[:, None], nx, axis=1))
        exact = (1.0 + 0.1 * k) * py[k] * (P(edges[1:]) - P(edges[:-1])) / dy
        np.testing.assert_allclose(LF[k][sl, 0], exact[sl], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("p_sign", [1, -1])
def test_linear_advection_2d_mode_along_y(oracle, p_sign):
    """The 2-D analogue of the Fourier-mode pin above, on the non-square box
    with periodic ghosts and no collisions: a mode along y of one population
    with p_x != 0 and p_y of either sign is multiplied in one step by the
    explicit stability function of (At, wt) at z = -dt |p_y|/dy sigma(theta)
    (1 - e^{-i theta}) (the x-sweep of an x-constant field is exactly 0)."""
    ny = BOX["ny"]
    pr = oracle.Problem(d=2, bc=1, Qphi=3, Qchi=1, gamma=1.4, tau=-1.0, dt=5e-3, **BOX)
    dy = (BOX["y1"] - BOX["y0"]) / ny
    theta = 2 * math.pi / 20
    s = np.arange(ny)
    c = np.array(golden("paper_values.json")["mp9"]["coefficients_over_2520"]) / 2520.0
    p, _ = oracle.gauss_hermite(3)
    At, _, wt, _ = _tab(oracle)
    k = (2 if p_sign > 0 else 0) * 3 + 2  # ky row of the requested sign, kx = 2 (p_x > 0)
    F0 = np.ones(pr.shape)
    F0[k] = (1.0 + 0.01 * np.cos(theta * s))[:, None]
    F1 = oracle.step(pr, F0, 1)
    pk = p[k // 3]
    th = theta if pk > 0 else -theta
    sigma = np.sum(c * np.exp(1j * th * np.arange(-4, 5)))
    eig = abs(pk) / dy * sigma * (1 - np.exp(-1j * th))
    R = _stability(At, wt, -pr.dt * eig)
    expect = 1.0 + 0.01 * np.real(R * np.exp(1j * theta * s))
    np.testing.assert_allclose(F1[k], np.repeat(expect[:, None], BOX["nx"], axis=1), rtol=0,
                               atol=1e-14)
    others = [j for j in range(pr.npop) if j != k]
    np.testing.assert_allclose(F1[others], 1.0, rtol=0, atol=1e-15)


# --------------------------------------------------------------------------
# Conservation and symmetries of the full step
# --------------------------------------------------------------------------

def _totals(oracle, pr, F):
    n, ux, uy, T = oracle.moments(pr, F)
    mass = n.sum()
    mom = (n * ux).sum()
    e = (n * (ux ** 2 + (uy ** 2 if uy is not None else 0)) + (2.0 / (pr.gamma - 1)) * n * T).sum()
    return np.array([mass, mom, e] + ([(n * uy).sum()] if uy is not None else []))


def test_conservation_periodic_1d(oracle):
    pr = oracle.Problem(d=1, nx=64, bc=1, Qphi=8, Qchi=8, gamma=1.4, tau=1e-4, dt=2e-3,
                        x0=0, x1=1)
    rho, u, T = W.smooth_fields_1d(64, seed=2, amp=0.2)
    F = oracle.init_fields(pr, rho, u, None, T)
    t0 = _totals(oracle, pr, F)
    G = oracle.step(pr, F, 50)
    t1 = _totals(oracle, pr, G)
    assert np.all(np.abs(t1 - t0) <= 1e-13 * np.maximum(1, np.abs(t0)) * 64), (t0, t1)


def test_conservation_periodic_2d(oracle):
    pr = oracle.Problem(d=2, nx=16, ny=16, bc=1, Qphi=5, Qchi=3, gamma=1.4, tau=1e-4, dt=4e-3,
                        x0=0, x1=1, y0=0, y1=1)
    rho, u, v, T = W.smooth_fields_2d(16, seed=4, amp=0.15)
    F = oracle.init_fields(pr, rho, u, v, T)
    t0 = _totals(oracle, pr, F)
    G = oracle.step(pr, F, 10)
    t1 = _totals(oracle, pr, G)
    assert np.all(np.abs(t1 - t0) <= 1e-13 * np.maximum(1, np.abs(t0)) * 256), (t0, t1)


def test_sod_outflow_momentum_balance(oracle):
    """Before any wave reaches the walls, mass and energy are constant and the
    total momentum grows by (P_L - P_R) t (outlet ghosts copy the wall cells)."""
    wl = W.sod_1d(nx=200, Q=8, tau=1e-6, dt=5e-5, t_end=0.05)
    pr = oracle.Problem(d=1, nx=wl.nx, x0=wl.x0, x1=wl.x1, Qphi=8, Qchi=8, gamma=1.4,
                        tau=wl.tau, dt=wl.dt)
    F = oracle.init_states(pr, wl.states, 0.0)
    ds = 1.0 / wl.nx
    t0 = _totals(oracle, pr, F) * ds
    G = oracle.step(pr, F, wl.nsteps)
    t1 = _totals(oracle, pr, G) * ds
    assert abs(t1[0] - t0[0]) < 1e-12
    assert abs(t1[2] - t0[2]) < 1e-12
    assert abs((t1[1] - t0[1]) - 0.9 * wl.t_end) < 1e-10


def test_mirror_symmetry_sod(oracle):
    # reflecting x -> -x (states swapped, velocities negated) reflects the solution
    pr = oracle.Problem(d=1, nx=100, Qphi=8, Qchi=8, gamma=1.4, tau=1e-6, dt=5e-5)
    L, R = (1.0, 0.2, 1.0), (0.125, -0.1, 0.1)
    F = oracle.init_states(pr, [L, R], 0.0)
    Fm = oracle.init_states(pr, [(R[0], -R[1], R[2]), (L[0], -L[1], L[2])], 0.0)
    G = oracle.step(pr, F, 100)
    Gm = oracle.step(pr, Fm, 100)
    n, u, _, T = oracle.moments(pr, G)
    nm, um, _, Tm = oracle.moments(pr, Gm)
    np.testing.assert_allclose(n, nm[::-1], rtol=1e-12)
    np.testing.assert_allclose(u, -um[::-1], rtol=0, atol=1e-12)
    np.testing.assert_allclose(T, Tm[::-1], rtol=1e-12)


def test_transpose_symmetry_2d(oracle):
    # swapping x and y (and u, v) transposes the 2-D solution
    pr = oracle.Problem(d=2, nx=20, ny=20, x0=0, x1=1, y0=0, y1=1, Qphi=5, Qchi=3, gamma=1.4,
                        tau=1e-5, dt=5e-4)
    st = np.array(W.C11_STATES)
    stT = st[[0, 3, 2, 1]][:, [0, 2, 1, 3]]  # quadrants 2 <-> 4, ux <-> uy
    F = oracle.init_states(pr, st, 0.5, 0.5)
    FT = oracle.init_states(pr, stT, 0.5, 0.5)
    G = oracle.step(pr, F, 10)
    GT = oracle.step(pr, FT, 10)
    n, ux, uy, T = oracle.moments(pr, G)
    nT, uxT, uyT, TT = oracle.moments(pr, GT)
    np.testing.assert_allclose(n, nT.T, rtol=1e-12)
    np.testing.assert_allclose(ux, uyT.T, rtol=0, atol=1e-12)
    np.testing.assert_allclose(T, TT.T, rtol=1e-12)


# --------------------------------------------------------------------------
# Sec. V: exact Riemann solution and the Sod comparison
# --------------------------------------------------------------------------

def test_exact_riemann_sod_textbook_values(oracle):
    g = golden("sod_star_textbook.json")
    xi = np.array([0.0])
    _, _, _, ps, us = oracle.riemann_exact(g["left"], g["right"], g["gamma"], xi)
    assert abs(ps - g["p_star"]) < g["abs_tol"]
    assert abs(us - g["u_star"]) < g["abs_tol"]
    # densities either side of the contact
    rl, _, _, _, _ = oracle.riemann_exact(g["left"], g["right"], g["gamma"], [us - 1e-9])
    rr, _, _, _, _ = oracle.riemann_exact(g["left"], g["right"], g["gamma"], [us + 1e-9])
    assert abs(rl[0] - g["rho_star_left"]) < g["abs_tol"]
    assert abs(rr[0] - g["rho_star_right"]) < g["abs_tol"]


def test_exact_riemann_rankine_hugoniot(oracle):
    """Across the Sod right-moving shock, mass, momentum and energy fluxes in the
    shock frame are continuous."""
    g, L, R = 1.4, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    xi = np.linspace(0.5, 2.5, 40001)
    rho, u, p, ps, us = oracle.riemann_exact(L, R, g, xi)
    jump = np.argmax(rho < 0.2)  # first sample in the undisturbed right state
    S = 0.5 * (xi[jump - 1] + xi[jump])
    r1, u1, p1 = rho[jump - 1], u[jump - 1], p[jump - 1]
    r2, u2, p2 = rho[jump], u[jump], p[jump]
    # shock speed from mass conservation
    S_mass = (r1 * u1 - r2 * u2) / (r1 - r2)
    assert abs(S_mass - S) < 1e-4
    E = lambda r, u, p: p / (g - 1) + 0.5 * r * u * u
    m1, m2 = r1 * (u1 - S_mass), r2 * (u2 - S_mass)
    assert abs(m1 - m2) < 1e-12
    assert abs((r1 * (u1 - S_mass) ** 2 + p1) - (r2 * (u2 - S_mass) ** 2 + p2)) < 1e-10
    f1 = (E(r1, u1, p1) + p1) * u1 - S_mass * E(r1, u1, p1)
    f2 = (E(r2, u2, p2) + p2) * u2 - S_mass * E(r2, u2, p2)
    assert abs(f1 - f2) < 1e-10


@pytest.mark.slow
def test_sod_l1_error_falls_with_resolution(oracle):
    """At tau << dt the scheme approaches the inviscid solution: L1(rho) against
    the exact Riemann solution decreases as S doubles (Sec. V)."""
    t_end = 0.1
    errs = []
    for nx in (100, 200, 400):
        wl = W.sod_1d(nx=nx, Q=8, tau=1e-6, dt=5e-5, t_end=t_end)
        pr = oracle.Problem(d=1, nx=nx, Qphi=8, Qchi=8, gamma=1.4, tau=wl.tau, dt=wl.dt)
        F = oracle.init_states(pr, wl.states, 0.0)
        G = oracle.step(pr, F, wl.nsteps)
        n, u, _, T = oracle.moments(pr, G)
        x = -0.5 + (np.arange(nx) + 0.5) / nx
        rho_ex, _, _, _, _ = oracle.riemann_exact(W.SOD_LEFT, W.SOD_RIGHT, 1.4, x / t_end)
        errs.append(np.mean(np.abs(n - rho_ex)))
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 6e-3, errs


@pytest.mark.slow
def test_time_order_three(oracle):
    """Smooth periodic flow at fixed grid, tau not stiff: halving dt divides the
    time-discretisation error by about 2^3 (IMEX-SSP3(4,3,3) is third order).
    Small single-mode perturbations of (rho, u, T), so that the MP limiter does
    not clip extrema (a clipped extremum makes the right-hand side only
    Lipschitz and lowers the observed order)."""
    nx = 32
    x = (np.arange(nx) + 0.5) / nx
    rho = 1 + 0.01 * np.sin(2 * np.pi * x)
    u = 0.01 * np.cos(2 * np.pi * x)
    T = 1 + 0.01 * np.sin(2 * np.pi * x + 1.0)
    t_end = 0.08
    sols = {}
    for m in (1, 2, 4, 32):
        dt = 4e-3 / m
        pr = oracle.Problem(d=1, nx=nx, bc=1, Qphi=8, Qchi=8, gamma=1.4, tau=0.02, dt=dt, x0=0, x1=1)
        F = oracle.init_fields(pr, rho, u, None, T)
        sols[m] = oracle.step(pr, F, int(round(t_end / dt)))
    e1 = np.abs(sols[1] - sols[32]).max()
    e2 = np.abs(sols[2] - sols[32]).max()
    e4 = np.abs(sols[4] - sols[32]).max()
    assert 6.5 < e1 / e2 < 10 and 6.5 < e2 / e4 < 10, (e1, e2, e4)


@pytest.mark.parametrize("S", [1, 2, 3, 4, 5, 7])
def test_periodic_ghosts_short_lines(oracle, S):
    """Periodic lines shorter than the 5-node halo: the advection of a line
    equals that of the same data repeated several times (the images of a
    periodic line are its cells taken modulo S)."""
    rng = np.random.default_rng(S)
    F = rng.uniform(0.5, 1.5, size=S)
    rep = 12
    for p in (1.3, -0.9):
        a = oracle.advect_line(F, p, 0.1, bc=1)
        b = oracle.advect_line(np.tile(F, rep), p, 0.1, bc=1)
        np.testing.assert_allclose(a, b[:S], rtol=0, atol=1e-14)
        np.testing.assert_allclose(a, b[S * (rep // 2):S * (rep // 2 + 1)], rtol=0, atol=1e-14)


def _sides(oracle, pr, states, xs, ys=0.5):
    """Which state each cell took: 1 where n is the second state's rho."""
    n = oracle.moments(pr, oracle.init_states(pr, states, xs, ys))[0]
    return n


@pytest.mark.parametrize("nx", [1, 3, 49, 103, 107, 755, 4095])
def test_membrane_on_a_cell_centre_takes_the_right_state(oracle, nx):
    """Sec. V set-up with an odd cell count and the membrane at the domain
    centre: the middle cell's centre lies exactly on it and it takes the right
    state; every cell left of it the left state.  (Comparing rounded centres
    x0 + (i + 1/2) dx with the membrane puts the middle cell on the left for
    49, 103, 107 and 275 of the 2048 odd lengths up to 4096.)"""
    pr = oracle.Problem(d=1, nx=nx, x0=-0.5, x1=0.5, Qphi=5, Qchi=3, gamma=1.4, tau=1e-5, dt=1e-5)
    n = _sides(oracle, pr, [[1.0, 0.0, 1.0], [0.25, 0.0, 0.3]], 0.0)
    mid = nx // 2
    assert np.allclose(n[mid:], 0.25, rtol=1e-14) and np.allclose(n[:mid], 1.0, rtol=1e-14)


def test_membrane_on_a_face_and_2d_centre(oracle):
    """Even cell count: the membrane at the centre lies on a face, cells
    nx/2 .. nx-1 are right of it.  2-D, 37 x 29 cells on [0, 1]^2 split at
    (0.5, 0.5): the middle row and column (centres on the membranes) belong
    to quadrant 1's side of each."""
    pr = oracle.Problem(d=1, nx=40, x0=-0.5, x1=0.5, Qphi=5, Qchi=3, gamma=1.4, tau=1e-5, dt=1e-5)
    n = _sides(oracle, pr, [[1.0, 0.0, 1.0], [0.25, 0.0, 0.3]], 0.0)
    assert np.allclose(n[20:], 0.25) and np.allclose(n[:20], 1.0)
    pr = oracle.Problem(d=2, nx=37, ny=29, x0=0.0, x1=1.0, y0=0.0, y1=1.0, Qphi=5, Qchi=3,
                        gamma=1.4, tau=1e-5, dt=1e-5)
    st = [[1.0, 0, 0, 1.0], [2.0, 0, 0, 1.0], [3.0, 0, 0, 1.0], [4.0, 0, 0, 1.0]]
    n = _sides(oracle, pr, st, 0.5, 0.5)
    want = np.empty((29, 37))
    want[14:, 18:], want[14:, :18], want[:14, :18], want[:14, 18:] = 1.0, 2.0, 3.0, 4.0
    assert np.allclose(n, want, rtol=1e-14)


def test_membrane_side_is_the_exact_comparison(oracle):
    """Seeded grids and membranes: a cell takes the right state exactly when
    its centre x0 + (i + 1/2)(x1 - x0)/nx, evaluated in rational arithmetic
    from the binary64 inputs, lies at or beyond the membrane."""
    from fractions import Fraction as Fr
    rng = np.random.default_rng(41)
    for _ in range(40):
        nx = int(rng.integers(1, 300))
        x0 = float(rng.uniform(-2.0, 0.0))
        x1 = x0 + float(rng.uniform(0.1, 3.0))
        xs = float(rng.uniform(x0 - 0.1, x1 + 0.1))
        pr = oracle.Problem(d=1, nx=nx, x0=x0, x1=x1, Qphi=3, Qchi=3, gamma=1.4, tau=1.0, dt=1e-9)
        n = _sides(oracle, pr, [[1.0, 0.0, 1.0], [0.25, 0.0, 0.3]], xs)
        want = [0.25 if Fr(x0) + (i + Fr(1, 2)) * (Fr(x1) - Fr(x0)) / nx >= Fr(xs) else 1.0
                for i in range(nx)]
        assert np.allclose(n, want, rtol=1e-14), (nx, x0, x1, xs)
