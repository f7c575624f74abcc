/*
 * fdlb_oracle.c -- plain, slow FP64 CPU oracle of the IMEX finite-difference
 * lattice Boltzmann method with reduced distributions (Kis & Ambrus, arXiv
 * 1909.08390).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the entry-point smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; everything below is
 * written from the paper's equations, in the paper's order:
 *
 *   Sec. II   Gauss-Hermite nodes/weights, Hermite-expanded equilibria
 *             (Eq. gExpanded), reduced distributions phi/chi (Eq. galpha),
 *             discrete moments (Eq. Moments_discrete);
 *   Sec. III  the general IMEX Runge-Kutta stage equation (Eq. IMEX) with the
 *             IMEX-SSP3(4,3,3) tableaux of Table I, each implicit stage solved
 *             in closed form because the collision term conserves the
 *             moments;
 *   Sec. IV   MP-9 interface values, the Suresh-Huynh MP limiter, flux
 *             differences, 5 ghost nodes per side with outlet conditions;
 *   Sec. V    piecewise-constant Riemann initial states and the analytic
 *             (exact) Riemann solution the Sod results are compared with.
 *
 * Built with -O2 -ffp-contract=off: every product and sum is rounded as
 * written.  Readings of passages where the paper is silent or garbled:
 *   - minmod of four arguments: common sign times the smallest magnitude when
 *     all four share a sign, else 0; sgn(0) = 0.
 *   - the MP flux is the unlimited F^L when (F^L-F_s)(F^L-F^MP) <= 0 (the
 *     paper gives only the strict cases); no epsilon.
 *   - negative velocity: the positive-velocity construction applied to the
 *     mirror image of the line (index s+j <-> s+1-j about each interface).
 *   - the interface value is multiplied by p to form the flux.
 *   - stage equations: the general Eq. (IMEX) with Table I (which makes the
 *     first stage F1 = F^n - alpha*dF1 and includes the (1-alpha)*dF2 term of
 *     stage 3 that the printed closed form of Eq. (IMEX_s34) drops).
 *   - initial populations are the discrete equilibria of the initial state.
 *   - D + K = 2/(gamma-1) with D = 3; only D+K and D+K-d enter.
 */
#include "fdlb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads.  The loops over cells, over (population, line) pairs and over
 * array elements are shared out with OpenMP; every output element is
 * computed by one thread with the same operations in the same order as on
 * one thread, so the results do not depend on the thread count. */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Sec. II: Gauss-Hermite quadrature                                         */
/* ------------------------------------------------------------------------ */

/* Probabilists' Hermite polynomial He_n(x) from the three-term recurrence
 * He_{k+1} = x He_k - k He_{k-1}, He_0 = 1, He_1 = x (the polynomials whose
 * roots are the lattice momenta, Sec. II). */
static long double he_ld(int n, long double x) {
  long double prev = 0.0L, cur = 1.0L;
  for (int k = 0; k < n; ++k) {
    long double next = x * cur - (long double)k * prev;
    prev = cur;
    cur = next;
  }
  return cur;
}

static long double fact_ld(int n) {
  long double f = 1.0L;
  for (int k = 2; k <= n; ++k) f *= (long double)k;
  return f;
}

/* Nodes p_k: the Q roots of He_Q, found by scanning for sign changes and
 * bisecting each bracket in long double.  Weights w_k = Q! / He_{Q+1}(p_k)^2
 * (Sec. II, the weight formula under Eq. Moments_discrete), which sum to 1. */
int orc_gauss_hermite(int Q, double* p, double* w) {
  if (Q < 1 || Q > ORC_MAXQ) return ORC_EINVAL;
  const long double L = sqrtl(4.0L * Q + 2.0L) + 1.0L; /* all roots lie inside */
  const int nscan = 20001;                             /* odd: 0 is not a grid point */
  const long double h = 2.0L * L / nscan;
  int found = 0;
  long double xa = -L, fa = he_ld(Q, xa);
  for (int i = 1; i <= nscan && found < Q; ++i) {
    long double xb = -L + h * i, fb = he_ld(Q, xb);
    if ((fa < 0.0L) != (fb < 0.0L)) {
      long double lo = xa, hi = xb, flo = fa;
      for (int it = 0; it < 400; ++it) {
        long double mid = 0.5L * (lo + hi);
        if (mid == lo || mid == hi) break;
        long double fm = he_ld(Q, mid);
        if (fm == 0.0L) { lo = hi = mid; break; }
        if ((fm < 0.0L) == (flo < 0.0L)) { lo = mid; flo = fm; } else { hi = mid; }
      }
      long double root = 0.5L * (lo + hi);
      /* He_Q is odd for odd Q, so x = 0 is then an exact root. */
      if ((Q % 2 == 1) && fabsl(root) < 1e-15L) root = 0.0L;
      p[found++] = (double)root;
    }
    xa = xb;
    fa = fb;
  }
  if (found != Q) return ORC_EINVAL;
  const long double qf = fact_ld(Q);
  for (int k = 0; k < Q; ++k) {
    long double hq1 = he_ld(Q + 1, (long double)p[k]);
    w[k] = (double)(qf / (hq1 * hq1));
  }
  return ORC_OK;
}

/* He_0(x) .. He_{Q-1}(x). */
void orc_he_values(int Q, double x, double* out) {
  for (int l = 0; l < Q; ++l) out[l] = (double)he_ld(l, (long double)x);
}

/* ------------------------------------------------------------------------ */
/* Sec. II, Eq. (gExpanded): Hermite-truncated one-axis equilibrium factor    */
/* ------------------------------------------------------------------------ */

static double ipow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

static double fact(int n) { return (double)fact_ld(n); }

/* Tables of one Gauss-Hermite axis used by the literal double sum below:
 * He_l(p_k) and l!/(2^s s! (l-2s)!) (computed once per lattice; the sum itself
 * is evaluated term by term in the order it is written). */
typedef struct {
  int Q;
  double p[ORC_MAXQ], w[ORC_MAXQ];
  double he[ORC_MAXQ][ORC_MAXQ];       /* he[k][l] = He_l(p_k) */
  double fl[ORC_MAXQ];                 /* l! */
  double coef[ORC_MAXQ][ORC_MAXQ / 2 + 1];
} axis_tab;

static void make_axis_tab(int Q, const double* p, const double* w, axis_tab* t) {
  t->Q = Q;
  for (int k = 0; k < Q; ++k) {
    t->p[k] = p[k];
    t->w[k] = w[k];
    orc_he_values(Q, p[k], t->he[k]);
  }
  for (int l = 0; l < Q; ++l) {
    t->fl[l] = fact(l);
    for (int s = 0; 2 * s <= l; ++s)
      t->coef[l][s] = fact(l) / (ipow(2.0, s) * fact(s) * fact(l - 2 * s));
  }
}

/* g^{Q-1}_k = w_k sum_{l=0}^{Q-1} He_l(p_k)/l! sum_{s=0}^{floor(l/2)}
 *             l!/(2^s s! (l-2s)!) (T-1)^s u^{l-2s}      (m = 1),
 * Eq. (gExpanded), evaluated literally as the double sum. */
static void g_axis_tab(const axis_tab* t, double u, double T, double* g) {
  const int Q = t->Q;
  double pt[ORC_MAXQ], pu[ORC_MAXQ]; /* (T-1)^e and u^e by repeated products */
  pt[0] = 1.0;
  pu[0] = 1.0;
  for (int e = 1; e < Q; ++e) {
    pt[e] = pt[e - 1] * (T - 1.0);
    pu[e] = pu[e - 1] * u;
  }
  for (int k = 0; k < Q; ++k) {
    double sum = 0.0;
    for (int l = 0; l < Q; ++l) {
      double inner = 0.0;
      for (int s = 0; 2 * s <= l; ++s) inner += t->coef[l][s] * pt[s] * pu[l - 2 * s];
      sum += t->he[k][l] / t->fl[l] * inner;
    }
    g[k] = t->w[k] * sum;
  }
}

void orc_g_axis(int Q, const double* p, const double* w, double u, double T, double* g) {
  axis_tab t;
  make_axis_tab(Q, p, w, &t);
  g_axis_tab(&t, u, T, g);
}

/* ------------------------------------------------------------------------ */
/* Table I: IMEX-SSP3(4,3,3)                                                  */
/* ------------------------------------------------------------------------ */

void orc_paper_tableau(orc_cfg* c) {
  const double al = 0.24169426078821, be = 0.06042356519705, et = 0.12915286960590;
  memset(c->At, 0, sizeof c->At);
  memset(c->A, 0, sizeof c->A);
  c->r = 4;
  /* explicit part */
  c->At[2][1] = 1.0;
  c->At[3][1] = 0.25;
  c->At[3][2] = 0.25;
  c->wt[0] = 0.0; c->wt[1] = 1.0 / 6.0; c->wt[2] = 1.0 / 6.0; c->wt[3] = 2.0 / 3.0;
  /* implicit part */
  c->A[0][0] = al;
  c->A[1][0] = -al; c->A[1][1] = al;
  c->A[2][1] = 1.0 - al; c->A[2][2] = al;
  c->A[3][0] = be; c->A[3][1] = et; c->A[3][2] = 0.5 - be - et - al; c->A[3][3] = al;
  c->w[0] = 0.0; c->w[1] = 1.0 / 6.0; c->w[2] = 1.0 / 6.0; c->w[3] = 2.0 / 3.0;
  c->alpha_mp = 4.0;
}

/* ------------------------------------------------------------------------ */
/* lattice helpers                                                            */
/* ------------------------------------------------------------------------ */

typedef struct {
  int d, Qp, Qc, nphi, nchi, P;
  double pp[ORC_MAXQ], wp[ORC_MAXQ]; /* phi nodes / weights */
  double pc[ORC_MAXQ], wc[ORC_MAXQ]; /* chi nodes / weights */
  double DK;                         /* D + K */
  axis_tab tp, tc;                   /* Eq. (gExpanded) tables, phi and chi axes */
} lattice;

static int make_lattice(const orc_cfg* c, lattice* L) {
  if (c->d < 1 || c->d > 2) return ORC_EINVAL;
  if (c->gamma <= 1.0) return ORC_EINVAL;
  L->d = c->d;
  L->Qp = c->Qphi;
  L->Qc = c->Qchi;
  if (orc_gauss_hermite(L->Qp, L->pp, L->wp)) return ORC_EINVAL;
  if (orc_gauss_hermite(L->Qc, L->pc, L->wc)) return ORC_EINVAL;
  L->nphi = L->Qp;
  L->nchi = L->Qc;
  if (c->d == 2) {
    L->nphi *= L->Qp;
    L->nchi *= L->Qc;
  }
  L->P = L->nphi + L->nchi;
  L->DK = 2.0 / (c->gamma - 1.0);
  if (L->DK - c->d < 0.0) return ORC_EINVAL;
  make_axis_tab(L->Qp, L->pp, L->wp, &L->tp);
  make_axis_tab(L->Qc, L->pc, L->wc, &L->tc);
  return ORC_OK;
}

int orc_npop(const orc_cfg* c) {
  lattice L;
  if (make_lattice(c, &L)) return ORC_EINVAL;
  return L.P;
}

/* momentum of phi population k along axis a (0 = x, 1 = y) */
static double phi_p(const lattice* L, int k, int a) {
  if (L->d == 1) return L->pp[k];
  return a == 0 ? L->pp[k % L->Qp] : L->pp[k / L->Qp];
}

/* ------------------------------------------------------------------------ */
/* Sec. II, Eq. (galpha) and Eq. (gExpanded): discrete equilibria             */
/* ------------------------------------------------------------------------ */

static void equilibrium_l(const lattice* L, double n, const double* u, double T, double* feq) {
  double gx[ORC_MAXQ], gy[ORC_MAXQ], hx[ORC_MAXQ], hy[ORC_MAXQ];
  /* phi^eq_k = n prod_a g_{a,k_a} */
  g_axis_tab(&L->tp, u[0], T, gx);
  if (L->d == 2) g_axis_tab(&L->tp, u[1], T, gy);
  for (int k = 0; k < L->nphi; ++k) {
    if (L->d == 1) feq[k] = n * gx[k];
    else feq[k] = n * gx[k % L->Qp] * gy[k / L->Qp];
  }
  /* chi^eq = (K + D - d) T phi^eq, expanded on the chi lattice */
  const double kchi = L->DK - L->d;
  g_axis_tab(&L->tc, u[0], T, hx);
  if (L->d == 2) g_axis_tab(&L->tc, u[1], T, hy);
  for (int q = 0; q < L->nchi; ++q) {
    double prod = (L->d == 1) ? hx[q] : hx[q % L->Qc] * hy[q / L->Qc];
    feq[L->nphi + q] = kchi * T * n * prod;
  }
}

int orc_equilibrium(const orc_cfg* c, double n, const double* u, double T, double* feq) {
  lattice L;
  if (make_lattice(c, &L)) return ORC_EINVAL;
  equilibrium_l(&L, n, u, T, feq);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. II, Eq. (Moments_discrete): n, u, T of one cell                       */
/* ------------------------------------------------------------------------ */

static int moments_l(const lattice* L, const double* F, long stride, double* n, double* u,
                     double* T) {
  double nn = 0.0, j[2] = {0.0, 0.0};
  for (int k = 0; k < L->nphi; ++k) {
    double f = F[k * stride];
    nn += f;
    for (int a = 0; a < L->d; ++a) j[a] += f * phi_p(L, k, a);
  }
  /* m = 1, so rho = n */
  for (int a = 0; a < L->d; ++a) u[a] = j[a] / nn;
  double e = 0.0; /* sum phi xi^2/2 + sum chi/2 = (D+K)/2 n T */
  for (int k = 0; k < L->nphi; ++k) {
    double xi2 = 0.0;
    for (int a = 0; a < L->d; ++a) {
      double xi = phi_p(L, k, a) - u[a];
      xi2 += xi * xi;
    }
    e += F[k * stride] * xi2 / 2.0;
  }
  for (int q = 0; q < L->nchi; ++q) e += F[(L->nphi + q) * stride] / 2.0;
  *n = nn;
  *T = 2.0 * e / (L->DK * nn);
  if (!(nn > 0.0) || !(*T > 0.0) || !isfinite(nn) || !isfinite(*T)) return ORC_EUNSTABLE;
  for (int a = 0; a < L->d; ++a)
    if (!isfinite(u[a])) return ORC_EUNSTABLE;
  return ORC_OK;
}

int orc_cell_moments(const orc_cfg* c, const double* F, long stride, double* n, double* u,
                     double* T) {
  lattice L;
  if (make_lattice(c, &L)) return ORC_EINVAL;
  return moments_l(&L, F, stride, n, u, T);
}

int orc_moments(const orc_cfg* c, const double* F, double* n, double* ux, double* uy, double* T) {
  lattice L;
  if (make_lattice(c, &L)) return ORC_EINVAL;
  const long N = (long)c->nx * (c->d == 2 ? c->ny : 1);
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(|| : bad)
  for (long i = 0; i < N; ++i) {
    double u[2] = {0.0, 0.0};
    int e = moments_l(&L, F + i, N, &n[i], u, &T[i]);
    if (e) bad = 1;
    ux[i] = u[0];
    if (uy) uy[i] = u[1];
  }
  return bad ? ORC_EUNSTABLE : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. IV: MP-9 interface value with the MP limiter (positive velocity)      */
/* ------------------------------------------------------------------------ */

static double sgn(double x) { return (double)((x > 0.0) - (x < 0.0)); }

/* minmod(x, y) = [sgn(x) + sgn(y)]/2 * min(|x|, |y|) */
static double minmod2(double x, double y) {
  return 0.5 * (sgn(x) + sgn(y)) * fmin(fabs(x), fabs(y));
}

/* four-argument minmod: common sign times the smallest magnitude, else 0 */
static double minmod4(double a, double b, double c, double d) {
  if (a > 0.0 && b > 0.0 && c > 0.0 && d > 0.0) return fmin(fmin(a, b), fmin(c, d));
  if (a < 0.0 && b < 0.0 && c < 0.0 && d < 0.0) return fmax(fmax(a, b), fmax(c, d));
  return 0.0;
}

static double min3(double a, double b, double c) { return fmin(a, fmin(b, c)); }
static double max3(double a, double b, double c) { return fmax(a, fmax(b, c)); }

/* v[0..8] = F_{s-4} .. F_{s+4}; returns the flux interface value at s+1/2 for
 * p > 0.  *limited (if non-NULL) is set when the limiter branch is taken. */
double orc_mp9_face(const double v[9], double alpha_mp, int* limited) {
  const double Fm2 = v[2], Fm1 = v[3], Fs = v[4], Fp1 = v[5], Fp2 = v[6];
  /* linear 9-point interface value */
  const double FL = (4.0 * v[0] - 41.0 * v[1] + 199.0 * v[2] - 641.0 * v[3] + 1879.0 * v[4] +
                     1375.0 * v[5] - 305.0 * v[6] + 55.0 * v[7] - 5.0 * v[8]) /
                    2520.0;
  /* monotonicity-preserving bound */
  const double FMP = Fs + minmod2(Fp1 - Fs, alpha_mp * (Fs - Fm1));
  if ((FL - Fs) * (FL - FMP) <= 0.0) {
    if (limited) *limited = 0;
    return FL;
  }
  if (limited) *limited = 1;
  /* curvatures C_s = F_{s+1} - 2 F_s + F_{s-1} */
  const double Cm1 = Fs - 2.0 * Fm1 + Fm2;
  const double C0 = Fp1 - 2.0 * Fs + Fm1;
  const double Cp1 = Fp2 - 2.0 * Fp1 + Fs;
  const double FUL = Fs + alpha_mp * (Fs - Fm1);
  const double FLC = Fs + 0.5 * (Fs - Fm1) +
                     (4.0 / 3.0) * minmod4(4.0 * C0 - Cm1, 4.0 * Cm1 - C0, C0, Cm1);
  const double FMD = 0.5 * (Fs + Fp1 - minmod4(4.0 * C0 - Cp1, 4.0 * Cp1 - C0, C0, Cp1));
  const double Fmin = fmax(min3(Fs, Fp1, FMD), min3(Fs, FUL, FLC));
  const double Fmax = fmin(max3(Fs, Fp1, FMD), max3(Fs, FUL, FLC));
  return FL + minmod2(Fmin - FL, Fmax - FL);
}

/* (p dF/dx)_s = p (Fhat_{s+1/2} - Fhat_{s-1/2}) / ds along one line of S
 * cells (element i at F[i*stride]); 5 ghost nodes per side: outlet copies of
 * the adjacent fluid node (bc 0) or periodic images (bc 1). */
void orc_advect_line(const double* F, int S, long stride, double p, double ds, int bc,
                     double alpha_mp, double* out, long ostride) {
  if (p == 0.0) {
    for (int s = 0; s < S; ++s) out[s * ostride] = 0.0;
    return;
  }
  double* ext = (double*)malloc(sizeof(double) * (size_t)(S + 10));
  double* face = (double*)malloc(sizeof(double) * (size_t)(S + 1));
  /* line as seen by a positive velocity: mirrored when p < 0 */
  for (int s = 0; s < S; ++s) {
    int src = (p > 0.0) ? s : S - 1 - s;
    ext[s + 5] = F[src * stride];
  }
  for (int g = 0; g < 5; ++g) {
    if (bc == 1) {
      /* periodic image of 0-based line position j is position j mod S */
      const int left = ((g - 5) % S + S) % S, right = (S + g) % S;
      ext[g] = ext[5 + left];
      ext[S + 5 + g] = ext[5 + right];
    } else {
      ext[g] = ext[5];
      ext[S + 5 + g] = ext[S + 4];
    }
  }
  /* face[s] is the interface between (1-based) cells s and s+1, s = 0..S;
   * its stencil F_{s-4..s+4} is ext[s .. s+8]. */
  for (int s = 0; s <= S; ++s) face[s] = orc_mp9_face(ext + s, alpha_mp, NULL);
  const double ap = fabs(p);
  for (int s = 0; s < S; ++s) {
    /* 0-based cell s is 1-based cell s+1: faces s+1 and s */
    double v = ap * (face[s + 1] - face[s]) / ds;
    int dst = (p > 0.0) ? s : S - 1 - s;
    out[dst * ostride] = v;
  }
  free(ext);
  free(face);
}

/* LF = p . grad F for every population (dimensionally unsplit: one 1-D MP-9
 * sweep per axis, the results summed). */
/* momentum of population k (phi or chi) along axis a */
static double pop_p(const lattice* L, int k, int a) {
  if (k < L->nphi) return (a == 1 && L->d == 1) ? 0.0 : phi_p(L, k, a);
  const int q = k - L->nphi;
  if (L->d == 1) return a == 0 ? L->pc[q] : 0.0;
  return a == 0 ? L->pc[q % L->Qc] : L->pc[q / L->Qc];
}

static void advect_l(const orc_cfg* c, const lattice* Lp, const double* F, double* LF) {
  const lattice L = *Lp;
  const int nx = c->nx, ny = (c->d == 2) ? c->ny : 1;
  const long N = (long)nx * ny;
  const double dx = (c->x1 - c->x0) / nx;
  const double dy = (c->d == 2) ? (c->y1 - c->y0) / ny : 1.0;
#pragma omp parallel
  {
    double* tmp = (double*)malloc(sizeof(double) * (size_t)(nx > ny ? nx : ny));
    /* x sweeps: line (k, y) starts row y of population k at 0 and adds its
     * flux differences */
#pragma omp for schedule(static)
    for (long kl = 0; kl < (long)L.P * ny; ++kl) {
      const int k = (int)(kl / ny), y = (int)(kl % ny);
      const double* Fk = F + (long)k * N;
      double* Lk = LF + (long)k * N;
      for (int x = 0; x < nx; ++x) Lk[(long)y * nx + x] = 0.0;
      orc_advect_line(Fk + (long)y * nx, nx, 1, pop_p(&L, k, 0), dx, c->bc, c->alpha_mp, tmp, 1);
      for (int x = 0; x < nx; ++x) Lk[(long)y * nx + x] += tmp[x];
    }
    /* y sweeps (after every x sweep: the loop above ends in a barrier) */
    if (L.d == 2) {
#pragma omp for schedule(static)
      for (long kl = 0; kl < (long)L.P * nx; ++kl) {
        const int k = (int)(kl / nx), x = (int)(kl % nx);
        const double* Fk = F + (long)k * N;
        double* Lk = LF + (long)k * N;
        orc_advect_line(Fk + x, ny, nx, pop_p(&L, k, 1), dy, c->bc, c->alpha_mp, tmp, 1);
        for (int y = 0; y < ny; ++y) Lk[(long)y * nx + x] += tmp[y];
      }
    }
    free(tmp);
  }
}

int orc_advect(const orc_cfg* c, const double* F, double* LF) {
  lattice L;
  if (make_lattice(c, &L)) return ORC_EINVAL;
  advect_l(c, &L, F, LF);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. V: initial states (F^0 = discrete equilibrium of the state)           */
/* ------------------------------------------------------------------------ */

/* 1-D: states[2][3] = (rho, u, P) left/right of xsplit.
 * 2-D: states[4][4] = (rho, ux, uy, P) of quadrants 1 (x>=xs, y>=ys),
 *      2 (x<xs, y>=ys), 3 (x<xs, y<ys), 4 (x>=xs, y<ys).
 * Cell centres x_s = x_left + (s - 1/2) ds; n = rho, T = P/rho (m = k_B = 1).
 * A cell whose centre lies on a membrane takes the right (upper) state.  The
 * test x_s >= xsplit is made in cell units, (s - 1/2) >= (xsplit - x_left)
 * nx / (x_right - x_left): that quotient is exact for a membrane at the
 * domain centre (nx/2), where rounded centres and a rounded ds would put the
 * middle cell of some odd nx on the left. */
int orc_init_states(const orc_cfg* c, const double* states, int nq, double xsplit,
                    double ysplit, double* F) {
  lattice L;
  if (make_lattice(c, &L)) return ORC_EINVAL;
  const int nx = c->nx, ny = (c->d == 2) ? c->ny : 1;
  const long N = (long)nx * ny;
  /* the membranes' positions in cells from the left (lower) edge */
  const double mx = (xsplit - c->x0) * (double)nx / (c->x1 - c->x0);
  const double my = (c->d == 2) ? (ysplit - c->y0) * (double)ny / (c->y1 - c->y0) : 0.0;
  if ((c->d == 1 && nq != 2) || (c->d == 2 && nq != 4)) return ORC_EINVAL;
  int bad = 0;
#pragma omp parallel reduction(|| : bad)
  {
  double* feq = (double*)malloc(sizeof(double) * (size_t)L.P);
#pragma omp for schedule(static)
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      const int right = (x + 0.5 >= mx);
      double rho, u[2] = {0.0, 0.0}, P;
      if (c->d == 1) {
        const double* s = states + 3 * right;
        rho = s[0]; u[0] = s[1]; P = s[2];
      } else {
        int quad;
        if (y + 0.5 >= my) quad = right ? 0 : 1;
        else quad = right ? 3 : 2;
        const double* s = states + 4 * quad;
        rho = s[0]; u[0] = s[1]; u[1] = s[2]; P = s[3];
      }
      if (!(rho > 0.0) || !(P > 0.0)) { bad = 1; continue; }
      equilibrium_l(&L, rho, u, P / rho, feq);
      for (int k = 0; k < L.P; ++k) F[(long)k * N + (long)y * nx + x] = feq[k];
    }
  }
  free(feq);
  }
  return bad ? ORC_EINVAL : ORC_OK;
}

/* Arbitrary per-cell (rho, u, T) fields, F = F_eq. */
int orc_init_fields(const orc_cfg* c, const double* rho, const double* ux, const double* uy,
                    const double* T, double* F) {
  lattice L;
  if (make_lattice(c, &L)) return ORC_EINVAL;
  const long N = (long)c->nx * (c->d == 2 ? c->ny : 1);
#pragma omp parallel
  {
    double* feq = (double*)malloc(sizeof(double) * (size_t)L.P);
#pragma omp for schedule(static)
    for (long i = 0; i < N; ++i) {
      double u[2] = {ux[i], (c->d == 2 && uy) ? uy[i] : 0.0};
      equilibrium_l(&L, rho[i], u, T[i], feq);
      for (int k = 0; k < L.P; ++k) F[(long)k * N + i] = feq[k];
    }
    free(feq);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. III, Eq. (IMEX): one IMEX Runge-Kutta step, general tableau form       */
/* ------------------------------------------------------------------------ */

/* For stage i:
 *   R_i   = F^n - dt sum_{j<i} At_ij L F^(j) - sum_{j<i} A_ij dF^(j)
 *   F^(i) = R_i - A_ii dF^(i),  dF^(i) = (dt/tau)(F^(i) - F^(i)_eq)
 * The collision term carries no mass, momentum or energy, so F^(i) has the
 * moments of R_i and F^(i)_eq is the equilibrium of those moments; the stage
 * is then linear in F^(i):
 *   F^(i) = (R_i + A_ii (dt/tau) F^(i)_eq) / (1 + A_ii dt/tau).
 * Finally F^{n+1} = F^n - dt sum_i wt_i L F^(i) - sum_i w_i dF^(i). */
int orc_step(const orc_cfg* c, double* F, int nsteps) {
  lattice L;
  if (make_lattice(c, &L)) return ORC_EINVAL;
  const int r = c->r;
  if (r < 1 || r > ORC_MAXR) return ORC_EINVAL;
  const long N = (long)c->nx * (c->d == 2 ? c->ny : 1);
  const long PN = (long)L.P * N;
  const double lam = (c->tau > 0.0) ? c->dt / c->tau : 0.0;
  int need_adv[ORC_MAXR];
  for (int j = 0; j < r; ++j) {
    need_adv[j] = (c->wt[j] != 0.0);
    for (int i = j + 1; i < r; ++i)
      if (c->At[i][j] != 0.0) need_adv[j] = 1;
  }
  double* Fi = (double*)malloc(sizeof(double) * (size_t)PN);
  double* R = (double*)malloc(sizeof(double) * (size_t)PN);
  double* LFs = (double*)calloc((size_t)r * (size_t)PN, sizeof(double));
  double* dFs = (double*)calloc((size_t)r * (size_t)PN, sizeof(double));
  if (!Fi || !R || !LFs || !dFs) {
    free(Fi); free(R); free(LFs); free(dFs);
    return ORC_ENOMEM;
  }
  int rc = ORC_OK;
  for (int step = 0; step < nsteps && rc == ORC_OK; ++step) {
    for (int i = 0; i < r && rc == ORC_OK; ++i) {
      /* explicit part */
#pragma omp parallel for schedule(static)
      for (long e = 0; e < PN; ++e) {
        double v = F[e];
        for (int j = 0; j < i; ++j) {
          v -= c->dt * c->At[i][j] * LFs[(long)j * PN + e];
          v -= c->A[i][j] * dFs[(long)j * PN + e];
        }
        R[e] = v;
      }
      /* implicit relaxation, cell by cell */
      const double aii = c->A[i][i];
      int bad = 0;
#pragma omp parallel reduction(|| : bad)
      {
        double* fq = (double*)malloc(sizeof(double) * (size_t)L.P);
#pragma omp for schedule(static)
        for (long cell = 0; cell < N; ++cell) {
          double n, u[2] = {0.0, 0.0}, T;
          if (moments_l(&L, R + cell, N, &n, u, &T)) { bad = 1; continue; }
          equilibrium_l(&L, n, u, T, fq);
          for (int k = 0; k < L.P; ++k) {
            const long idx = (long)k * N + cell;
            const double fi = (R[idx] + aii * lam * fq[k]) / (1.0 + aii * lam);
            Fi[idx] = fi;
            dFs[(long)i * PN + idx] = lam * (fi - fq[k]);
          }
        }
        free(fq);
      }
      if (bad) { rc = ORC_EUNSTABLE; break; }
      if (need_adv[i]) advect_l(c, &L, Fi, LFs + (long)i * PN);
    }
    if (rc) break;
    int nonfinite = 0;
#pragma omp parallel for schedule(static) reduction(|| : nonfinite)
    for (long e = 0; e < PN; ++e) {
      double v = F[e];
      for (int i = 0; i < r; ++i) {
        v -= c->dt * c->wt[i] * LFs[(long)i * PN + e];
        v -= c->w[i] * dFs[(long)i * PN + e];
      }
      if (!isfinite(v)) nonfinite = 1;
      F[e] = v;
    }
    if (nonfinite) rc = ORC_EUNSTABLE;
  }
  free(Fi); free(R); free(LFs); free(dFs);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. V: exact solution of the Riemann problem of the Euler equations        */
/* (the analytic Sod solution the paper compares with), ideal gas gamma.      */
/* ------------------------------------------------------------------------ */

/* Velocity jump across the left or right wave as a function of the star
 * pressure: Rankine-Hugoniot shock (p > pK) or isentropic rarefaction. */
static double wave_fn(double p, double rhoK, double pK, double g) {
  const double cK = sqrt(g * pK / rhoK);
  if (p > pK) {
    const double A = 2.0 / ((g + 1.0) * rhoK), B = (g - 1.0) / (g + 1.0) * pK;
    return (p - pK) * sqrt(A / (p + B));
  }
  return 2.0 * cK / (g - 1.0) * (pow(p / pK, (g - 1.0) / (2.0 * g)) - 1.0);
}

int orc_riemann_exact(double rhoL, double uL, double pL, double rhoR, double uR, double pR,
                      double g, const double* xi, int n, double* rho, double* u, double* p,
                      double* pstar, double* ustar) {
  const double cL = sqrt(g * pL / rhoL), cR = sqrt(g * pR / rhoR);
  const double du = uR - uL;
  /* vacuum generation: no positive star pressure */
  if (2.0 * (cL + cR) / (g - 1.0) <= du) return ORC_EINVAL;
  /* f(p) = fL(p) + fR(p) + du is increasing in p: bracket then bisect */
  double lo = 0.0, hi = fmax(pL, pR);
  while (wave_fn(hi, rhoL, pL, g) + wave_fn(hi, rhoR, pR, g) + du < 0.0) hi *= 2.0;
  for (int it = 0; it < 2000; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    double f = wave_fn(mid, rhoL, pL, g) + wave_fn(mid, rhoR, pR, g) + du;
    if (f < 0.0) lo = mid; else hi = mid;
  }
  const double ps = 0.5 * (lo + hi);
  const double us = 0.5 * (uL + uR) + 0.5 * (wave_fn(ps, rhoR, pR, g) - wave_fn(ps, rhoL, pL, g));
  if (pstar) *pstar = ps;
  if (ustar) *ustar = us;
  const double gm = (g - 1.0) / (g + 1.0);
  for (int i = 0; i < n; ++i) {
    const double s = xi[i];
    double r_, u_, p_;
    if (s <= us) {
      if (ps > pL) { /* left shock */
        const double SL = uL - cL * sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g));
        if (s < SL) { r_ = rhoL; u_ = uL; p_ = pL; }
        else { r_ = rhoL * (ps / pL + gm) / (gm * ps / pL + 1.0); u_ = us; p_ = ps; }
      } else { /* left rarefaction */
        const double cs = cL * pow(ps / pL, (g - 1.0) / (2.0 * g));
        const double head = uL - cL, tail = us - cs;
        if (s < head) { r_ = rhoL; u_ = uL; p_ = pL; }
        else if (s > tail) { r_ = rhoL * pow(ps / pL, 1.0 / g); u_ = us; p_ = ps; }
        else {
          u_ = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL + s);
          const double cc = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * (uL - s));
          r_ = rhoL * pow(cc / cL, 2.0 / (g - 1.0));
          p_ = pL * pow(cc / cL, 2.0 * g / (g - 1.0));
        }
      }
    } else {
      if (ps > pR) { /* right shock */
        const double SR = uR + cR * sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g));
        if (s > SR) { r_ = rhoR; u_ = uR; p_ = pR; }
        else { r_ = rhoR * (ps / pR + gm) / (gm * ps / pR + 1.0); u_ = us; p_ = ps; }
      } else { /* right rarefaction */
        const double cs = cR * pow(ps / pR, (g - 1.0) / (2.0 * g));
        const double head = uR + cR, tail = us + cs;
        if (s > head) { r_ = rhoR; u_ = uR; p_ = pR; }
        else if (s < tail) { r_ = rhoR * pow(ps / pR, 1.0 / g); u_ = us; p_ = ps; }
        else {
          u_ = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * uR + s);
          const double cc = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * (uR - s));
          r_ = rhoR * pow(cc / cR, 2.0 / (g - 1.0));
          p_ = pR * pow(cc / cR, 2.0 * g / (g - 1.0));
        }
      }
    }
    rho[i] = r_;
    u[i] = u_;
    p[i] = p_;
  }
  return ORC_OK;
}
