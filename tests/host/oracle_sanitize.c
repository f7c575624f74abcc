/* Driver of the CPU oracle (oracle/fdlb_oracle.c) for the address and
 * undefined-behaviour sanitizers: every entry point on small and degenerate
 * sizes (single cells, lines shorter than the 5-node ghost layers, odd 2-D
 * shapes), both boundaries, three lattices, rejected arguments.  Exits
 * non-zero on any unexpected return code; the sanitizers abort on any
 * out-of-bounds access, use after free, leak or undefined operation. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "../../oracle/fdlb_oracle.h"

static int fails = 0;
#define EXPECT(cond)                                            \
  do {                                                          \
    if (!(cond)) {                                              \
      fprintf(stderr, "%s:%d: %s\n", __FILE__, __LINE__, #cond); \
      ++fails;                                                  \
    }                                                           \
  } while (0)

static double urand(unsigned* s) {
  *s = *s * 1664525u + 1013904223u;
  return (double)(*s >> 8) / 16777216.0;
}

static void run_problem(int d, int nx, int ny, int bc, int Qp, int Qc, int steps) {
  orc_cfg c = {0};
  c.d = d;
  c.nx = nx;
  c.ny = d == 2 ? ny : 1;
  c.x0 = 0.0;
  c.x1 = 1.0;
  c.y0 = 0.0;
  c.y1 = 0.7;
  c.bc = bc;
  c.Qphi = Qp;
  c.Qchi = Qc;
  c.gamma = 1.4;
  c.tau = 1e-4;
  c.dt = 2e-4;
  orc_paper_tableau(&c);
  const int P = orc_npop(&c);
  EXPECT(P == (d == 1 ? Qp + Qc : Qp * Qp + Qc * Qc));
  const long N = (long)nx * c.ny;
  double* F = malloc(sizeof(double) * (size_t)(P * N));
  double* LF = malloc(sizeof(double) * (size_t)(P * N));
  double* m = malloc(sizeof(double) * (size_t)(4 * N));
  const double st1[6] = {1.0, 0.1, 1.0, 0.5, -0.2, 0.4};
  const double st2[16] = {1.0, 0.1, 0.0, 1.0, 0.5, 0.8, 0.0, 0.4,
                          0.8, 0.1, 0.0, 0.4, 0.5, 0.1, 0.7, 0.4};
  EXPECT(orc_init_states(&c, d == 1 ? st1 : st2, d == 1 ? 2 : 4, 0.5, 0.35, F) == ORC_OK);
  EXPECT(orc_advect(&c, F, LF) == ORC_OK);
  EXPECT(orc_step(&c, F, steps) == ORC_OK);
  EXPECT(orc_moments(&c, F, m, m + N, d == 2 ? m + 2 * N : NULL, m + 3 * N) == ORC_OK);
  /* fields */
  for (long i = 0; i < N; ++i) {
    m[i] = 1.0 + 0.1 * (double)(i % 3);
    m[N + i] = 0.05;
    m[2 * N + i] = -0.05;
    m[3 * N + i] = 0.9;
  }
  EXPECT(orc_init_fields(&c, m, m + N, d == 2 ? m + 2 * N : NULL, m + 3 * N, F) == ORC_OK);
  /* a cell with n < 0 is reported, not crashed on */
  for (int k = 0; k < P; ++k) F[(long)k * N] = -1.0;
  EXPECT(orc_moments(&c, F, m, m + N, d == 2 ? m + 2 * N : NULL, m + 3 * N) == ORC_EUNSTABLE);
  EXPECT(orc_step(&c, F, 1) == ORC_EUNSTABLE);
  free(F);
  free(LF);
  free(m);
}

int main(void) {
  orc_set_threads(2);
  /* quadrature and equilibrium factors */
  double p[ORC_MAXQ], w[ORC_MAXQ], g[ORC_MAXQ], he[ORC_MAXQ];
  for (int Q = 1; Q <= ORC_MAXQ; ++Q) {
    EXPECT(orc_gauss_hermite(Q, p, w) == ORC_OK);
    orc_g_axis(Q, p, w, 0.3, 1.2, g);
    orc_he_values(Q, p[0], he);
  }
  EXPECT(orc_gauss_hermite(0, p, w) == ORC_EINVAL);
  EXPECT(orc_gauss_hermite(ORC_MAXQ + 1, p, w) == ORC_EINVAL);
  /* MP-9 interface values on random windows */
  unsigned s = 12345u;
  for (int t = 0; t < 2000; ++t) {
    double v[9];
    for (int j = 0; j < 9; ++j) v[j] = urand(&s) - 0.5;
    int lim = 0;
    const double f = orc_mp9_face(v, 4.0, &lim);
    EXPECT(isfinite(f));
  }
  /* lines shorter than, equal to and longer than the ghost layers */
  for (int S = 1; S <= 13; ++S)
    for (int bc = 0; bc < 2; ++bc) {
      double line[13], out[13];
      for (int i = 0; i < S; ++i) line[i] = 1.0 + urand(&s);
      orc_advect_line(line, S, 1, 1.3, 0.1, bc, 4.0, out, 1);
      orc_advect_line(line, S, 1, -0.7, 0.1, bc, 4.0, out, 1);
      orc_advect_line(line, S, 1, 0.0, 0.1, bc, 4.0, out, 1);
    }
  /* whole steps */
  const int lat[3][2] = {{3, 3}, {5, 3}, {8, 8}};
  for (int l = 0; l < 3; ++l)
    for (int bc = 0; bc < 2; ++bc) {
      run_problem(1, 1, 1, bc, lat[l][0], lat[l][1], 2);
      run_problem(1, 7, 1, bc, lat[l][0], lat[l][1], 2);
      run_problem(2, 1, 1, bc, lat[l][0], lat[l][1], 1);
      run_problem(2, 3, 5, bc, lat[l][0], lat[l][1], 1);
      run_problem(2, 7, 4, bc, lat[l][0], lat[l][1], 1);
    }
  /* rejected configurations */
  orc_cfg bad = {0};
  bad.d = 3;
  bad.nx = bad.ny = 4;
  bad.Qphi = bad.Qchi = 3;
  bad.gamma = 1.4;
  EXPECT(orc_npop(&bad) == ORC_EINVAL);
  bad.d = 2;
  bad.gamma = 3.0; /* D + K - d < 0 */
  EXPECT(orc_npop(&bad) == ORC_EINVAL);
  /* exact Riemann solution, including a vacuum-generating pair */
  double xi[5] = {-2.0, -0.5, 0.0, 0.5, 2.0}, r[5], u[5], pp[5], ps, us;
  EXPECT(orc_riemann_exact(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4, xi, 5, r, u, pp, &ps, &us) ==
         ORC_OK);
  EXPECT(orc_riemann_exact(1.0, -20.0, 1.0, 1.0, 20.0, 1.0, 1.4, xi, 5, r, u, pp, &ps, &us) ==
         ORC_EINVAL);
  if (fails) fprintf(stderr, "%d failed expectations\n", fails);
  else printf("oracle sanitize driver: ok\n");
  return fails ? 1 : 0;
}
