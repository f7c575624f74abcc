/*
 * fdlb_oracle.h -- plain FP64 CPU oracle of the IMEX finite-difference lattice
 * Boltzmann step (Kis & Ambrus, "Implicit-Explicit Finite-Difference Lattice
 * Boltzmann Model with Varying Adiabatic Index").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the tests, the entry-point smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * constant with the CUDA library.
 *
 * Layout convention (the only thing the two sides have to agree on, since the
 * parity tests compare arrays element by element):
 *   state F[P][ny][nx] (x fastest; 1-D: ny = 1), P = Qphi^d + Qchi^d;
 *   populations 0 .. Qphi^d-1 are phi_k with k = ky*Qphi + kx (1-D: k = kx),
 *   populations Qphi^d .. P-1 are chi_q with q = qy*Qchi + qx;
 *   velocity nodes in ascending order of p.
 */
#ifndef FDLB_ORACLE_H
#define FDLB_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXQ 16
#define ORC_MAXR 8

typedef struct {
  int d;              /* number of inhomogeneous axes, 1 or 2 */
  int nx, ny;         /* cells per axis (ny = 1 when d = 1) */
  double x0, x1;      /* domain along x */
  double y0, y1;      /* domain along y (ignored when d = 1) */
  int bc;             /* 0 outflow (ghosts copy the adjacent fluid node), 1 periodic */
  int Qphi, Qchi;     /* Gauss-Hermite orders per axis */
  double gamma;       /* adiabatic index; D + K = 2/(gamma - 1) */
  double tau, dt;     /* relaxation time, time step; tau <= 0 means no collision */
  int r;              /* number of IMEX stages */
  double At[ORC_MAXR][ORC_MAXR], A[ORC_MAXR][ORC_MAXR];
  double wt[ORC_MAXR], w[ORC_MAXR];
  double alpha_mp;    /* MP limiter coefficient (4 in the paper) */
} orc_cfg;

/* error codes */
#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_EUNSTABLE -5
#define ORC_ENOMEM -3

/* Threads of the oracle's loops (OpenMP): n > 0 sets the count, n <= 0
 * keeps it; returns the count the loops use.  Results do not depend on it. */
int orc_set_threads(int n);
int orc_gauss_hermite(int Q, double* p, double* w);
void orc_he_values(int Q, double x, double* out);
void orc_g_axis(int Q, const double* p, const double* w, double u, double T, double* g);
void orc_paper_tableau(orc_cfg* c);
int orc_npop(const orc_cfg* c);
int orc_equilibrium(const orc_cfg* c, double n, const double* u, double T, double* feq);
int orc_cell_moments(const orc_cfg* c, const double* F, long stride, double* n, double* u, double* T);
int orc_moments(const orc_cfg* c, const double* F, double* n, double* ux, double* uy, double* T);
double orc_mp9_face(const double v[9], double alpha_mp, int* limited);
void orc_advect_line(const double* F, int S, long stride, double p, double ds, int bc,
                     double alpha_mp, double* out, long ostride);
int orc_advect(const orc_cfg* c, const double* F, double* LF);
int orc_init_states(const orc_cfg* c, const double* states, int nq, double xsplit,
                    double ysplit, double* F);
int orc_init_fields(const orc_cfg* c, const double* rho, const double* ux, const double* uy,
                    const double* T, double* F);
int orc_step(const orc_cfg* c, double* F, int nsteps);
int orc_riemann_exact(double rhoL, double uL, double pL, double rhoR, double uR, double pR,
                      double gamma, const double* xi, int n, double* rho, double* u, double* p,
                      double* pstar, double* ustar);

#ifdef __cplusplus
}
#endif
#endif
