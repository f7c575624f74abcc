// fdlb_api.cpp -- host side of libfdlb.so: the C ABI declared in
// include/fdlb.h, lattice construction, validation and stage coefficients.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <algorithm>

#include "fdlb.h"
#include "fdlb_ctx.h"
#include "fdlb_internal.h"

using fdlb::DevParams;
using fdlb::kMaxQ;


namespace {

std::string g_create_error = "no error";

int set_err(fdlb_ctx* c, int code, const char* fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof msg, fmt, ap);
  va_end(ap);
  if (c) c->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_err(fdlb_ctx* c, cudaError_t e, const char* what) {
  return set_err(c, FDLB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// He_n(x) (probabilists') and He_n'(x) = n He_{n-1}(x) by the recurrence
// He_{k+1} = x He_k - k He_{k-1}.
void hermite(int n, long double x, long double* h, long double* dh) {
  long double hm1 = 0.0L, h0 = 1.0L;
  for (int k = 0; k < n; ++k) {
    long double hp = x * h0 - (long double)k * hm1;
    hm1 = h0;
    h0 = hp;
  }
  *h = h0;
  *dh = (long double)n * hm1;
}

// Gauss-Hermite rule for the weight exp(-p^2/2)/sqrt(2 pi): the Q roots of
// He_Q by simultaneous Newton (Ehrlich-Aberth) iteration from Chebyshev-spaced
// starting points, then exact antisymmetry p_{Q-1-k} = -p_k, and weights
// w_k = Q!/He_{Q+1}(p_k)^2 (Sec. II).
bool gauss_hermite(int Q, double* p_out, double* w_out) {
  if (Q < 1 || Q > kMaxQ) return false;
  long double z[kMaxQ];
  const long double R = sqrtl(4.0L * Q + 2.0L);
  for (int i = 0; i < Q; ++i)
    z[i] = -R * cosl(3.14159265358979323846L * (i + 0.5L) / Q) * 0.9L;
  for (int it = 0; it < 500; ++it) {
    long double maxstep = 0.0L;
    for (int i = 0; i < Q; ++i) {
      long double h, dh;
      hermite(Q, z[i], &h, &dh);
      if (h == 0.0L) continue;
      const long double ratio = h / dh;
      long double s = 0.0L;
      for (int j = 0; j < Q; ++j)
        if (j != i) s += 1.0L / (z[i] - z[j]);
      const long double step = ratio / (1.0L - ratio * s);
      z[i] -= step;
      if (fabsl(step) > maxstep) maxstep = fabsl(step);
    }
    if (maxstep < 1e-30L) break;
  }
  // sort ascending (insertion sort) and enforce p(-x) symmetry
  for (int i = 1; i < Q; ++i)
    for (int j = i; j > 0 && z[j] < z[j - 1]; --j) {
      long double t = z[j];
      z[j] = z[j - 1];
      z[j - 1] = t;
    }
  for (int i = 0; i < Q / 2; ++i) {
    const long double a = 0.5L * (z[Q - 1 - i] - z[i]);
    z[i] = -a;
    z[Q - 1 - i] = a;
  }
  if (Q % 2 == 1) z[Q / 2] = 0.0L;
  long double qf = 1.0L;
  for (int k = 2; k <= Q; ++k) qf *= (long double)k;
  for (int i = 0; i < Q; ++i) {
    long double h, dh;
    hermite(Q + 1, z[i], &h, &dh);
    p_out[i] = (double)z[i];
    w_out[i] = (double)(qf / (h * h));
  }
  // converged: the Newton correction at every root is below 1e-15 (1 + |p|)
  for (int i = 0; i < Q; ++i) {
    long double h, dh;
    hermite(Q, z[i], &h, &dh);
    if (!(fabsl(h / dh) <= 1e-15L * (1.0L + fabsl(z[i])))) return false;
  }
  return true;
}

// wH[l*kMaxQ + k] = w_k He_l(p_k) / l!
void weighted_hermite_table(int Q, const double* p, const double* w, double* wH) {
  for (int k = 0; k < Q; ++k) {
    long double hm1 = 0.0L, h0 = 1.0L, fl = 1.0L;
    for (int l = 0; l < Q; ++l) {
      if (l > 0) fl *= (long double)l;
      wH[l * kMaxQ + k] = (double)((long double)w[k] * h0 / fl);
      long double hp = (long double)p[k] * h0 - (long double)l * hm1;
      hm1 = h0;
      h0 = hp;
    }
  }
}

void paper_tableau(fdlb_tableau* t) {
  // Table I: IMEX-SSP3(4,3,3)
  const double al = 0.24169426078821, be = 0.06042356519705, et = 0.12915286960590;
  std::memset(t, 0, sizeof *t);
  t->r = 4;
  t->At[2 * 4 + 1] = 1.0;
  t->At[3 * 4 + 1] = 0.25;
  t->At[3 * 4 + 2] = 0.25;
  t->A[0 * 4 + 0] = al;
  t->A[1 * 4 + 0] = -al;
  t->A[1 * 4 + 1] = al;
  t->A[2 * 4 + 1] = 1.0 - al;
  t->A[2 * 4 + 2] = al;
  t->A[3 * 4 + 0] = be;
  t->A[3 * 4 + 1] = et;
  t->A[3 * 4 + 2] = 0.5 - be - et - al;
  t->A[3 * 4 + 3] = al;
  t->wt[1] = t->wt[2] = 1.0 / 6.0;
  t->wt[3] = 2.0 / 3.0;
  t->w[1] = t->w[2] = 1.0 / 6.0;
  t->w[3] = 2.0 / 3.0;
}

// Reduce a supported tableau to the fused-stage coefficients (see
// fdlb_internal.h for the algebra).
// Shu-Osher SSP-RK3 on the whole right-hand side: stages F^n, F^n,
// F^n + dt f(F^n), F^n + dt (f(F^n) + f(F^(3)))/4; weights (0, 1/6, 1/6, 2/3).
void explicit_ssprk3_tableau(fdlb_tableau* t) {
  std::memset(t, 0, sizeof *t);
  t->r = 4;
  t->At[2 * 4 + 1] = t->A[2 * 4 + 1] = 1.0;
  t->At[3 * 4 + 1] = t->A[3 * 4 + 1] = 0.25;
  t->At[3 * 4 + 2] = t->A[3 * 4 + 2] = 0.25;
  t->wt[1] = t->wt[2] = t->w[1] = t->w[2] = 1.0 / 6.0;
  t->wt[3] = t->w[3] = 2.0 / 3.0;
}

bool stage_coefficients(const fdlb_tableau& t, double lam, fdlb::StageCoef* sc, const char** why) {
  if (t.r != 4) { *why = "the fused kernels need r = 4 stages"; return false; }
  auto At = [&](int i, int j) { return t.At[i * 4 + j]; };
  auto A = [&](int i, int j) { return t.A[i * 4 + j]; };
  for (int i = 0; i < 4; ++i) {
    if (At(i, 0) != 0.0) { *why = "stage 1 must not be advected (At[i][0] = 0)"; return false; }
    for (int j = i; j < 4; ++j)
      if (At(i, j) != 0.0) { *why = "At must be strictly lower triangular"; return false; }
    for (int j = i + 1; j < 4; ++j)
      if (A(i, j) != 0.0) { *why = "A must be lower triangular"; return false; }
  }
  if (t.wt[0] != 0.0) { *why = "wt[0] must be 0"; return false; }
  double e[4];
  for (int i = 0; i < 4; ++i) {
    const double den = 1.0 + A(i, i) * lam;
    if (!(den > 0.0)) { *why = "1 + a_ii dt/tau must be positive"; return false; }
    e[i] = lam / den;
  }
  // dF1 = e1 D; R2 = F - a21 dF1, dF2 = e2 (1 - a21 e1) D; F2 = F - a21 dF1 - a22 dF2
  const double d1 = e[0];
  const double d2 = e[1] * (1.0 - A(1, 0) * d1);
  sc->c2 = 1.0 - A(1, 0) * d1 - A(1, 1) * d2;
  sc->k3 = A(2, 0) * d1 + A(2, 1) * d2;
  sc->k4 = A(3, 0) * d1 + A(3, 1) * d2;
  sc->kf = t.w[0] * d1 + t.w[1] * d2;
  sc->at32 = At(2, 1);
  sc->at42 = At(3, 1);
  sc->at43 = At(3, 2);
  sc->wt2 = t.wt[1];
  sc->wt3 = t.wt[2];
  sc->wt4 = t.wt[3];
  sc->a33e3 = A(2, 2) * e[2];
  sc->a43e3 = A(3, 2) * e[2];
  sc->w3e3 = t.w[2] * e[2];
  sc->a44e4 = A(3, 3) * e[3];
  sc->w4e4 = t.w[3] * e[3];
  return true;
}

// x = hi + lo with hi = binary32(x) and lo = binary32(x - hi): 48 of x's 53
// significant bits, for the compensated binary32 moment sums.
void split_float(double x, float* hi, float* lo) {
  *hi = (float)x;
  *lo = (float)(x - (double)*hi);
}

// One stage of a context: the grid-mapped kernels of a single problem or the
// persistent work-list kernels of a batch.
int launch_stage_any(const fdlb_ctx* c, int stage, cudaStream_t s) {
  return c->batch ? fdlb::launch_batch_stage(c->dp, stage, s) : fdlb::launch_stage(c->dp, stage, s);
}

constexpr int kGraphSteps = 16;  // steps per captured graph (even: see step_launch)

// Point the stage kernels of a FDLB_MIXED context at the current state buffer
// (pair[parity]) and the one the final stage writes.
void set_pair_pointers(fdlb_ctx* c) {
  if (c->precision != FDLB_MIXED) return;
  c->dp.sh = c->pair[c->parity][0];
  c->dp.sl = c->pair[c->parity][1];
  c->dp.nh = c->pair[1 - c->parity][0];
  c->dp.nl = c->pair[1 - c->parity][1];
}

// One stage kernel of a step; after the final stage of a FDLB_MIXED context
// the new state is in the other buffer, which becomes the current one.
int step_launch(fdlb_ctx* c, int stage, cudaStream_t s) {
  const int e = launch_stage_any(c, stage, s);
  if (!e && stage == fdlb::kFinal && c->precision == FDLB_MIXED) {
    c->parity ^= 1;
    set_pair_pointers(c);
  }
  return e;
}

void drop_graph(fdlb_ctx* c) {
  for (auto& g : c->graph_exec) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
}

// Capture kGraphSteps steps (3 kernels each) on a private stream once per
// starting state buffer; the graph then replays on the context's stream.
// kGraphSteps is even, so a replay ends in the buffer it started from.
int ensure_graph(fdlb_ctx* c) {
  if (c->graph_exec[c->parity]) return FDLB_OK;
  const int start_parity = c->parity;
  cudaError_t e = cudaSuccess;
  if (!c->capture_stream) e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_err(c, e, "capture stream");
  e = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_err(c, e, "cudaStreamBeginCapture");
  int le = 0;
  for (int k = 0; k < kGraphSteps && !le; ++k)
    for (int st : {fdlb::kStage3, fdlb::kStage4, fdlb::kFinal})
      if (!le) le = step_launch(c, st, c->capture_stream);
  // the capture ran nothing: the state is where it was
  c->parity = start_parity;
  set_pair_pointers(c);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(c->capture_stream, &g);
  if (le) {
    if (g) cudaGraphDestroy(g);
    return cuda_err(c, (cudaError_t)le, "kernel launch during capture");
  }
  if (e != cudaSuccess) return cuda_err(c, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&c->graph_exec[start_parity], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->graph_exec[start_parity] = nullptr;
    return cuda_err(c, e, "cudaGraphInstantiate");
  }
  return FDLB_OK;
}

// Device buffers of a context: FDLB_FP64, six binary64 population arrays
// (F, F2, F3, A4, A_fin, D); FDLB_MIXED, eleven binary32 population arrays
// (the two state buffers hi and lo, r3l, a4l, afl, dm, fa, fb, fc) and the
// per-cell mhi; then the four moment fields for host copies and the status
// word.
struct Layout {
  size_t arr, mom, mhi, total;
};

Layout buffer_layout(int precision, int P, int64_t N) {
  Layout L{};
  const size_t esize = precision == FDLB_MIXED ? sizeof(float) : sizeof(double);
  L.arr = ((size_t)P * (size_t)N * esize + 255) / 256 * 256;
  const size_t narr = precision == FDLB_MIXED ? 11 : 6;
  L.mom = narr * L.arr;
  L.mhi = L.mom + 4 * (size_t)N * sizeof(double) + 256;
  L.total = L.mhi + (precision == FDLB_MIXED ? 4 * (size_t)N * sizeof(double) : 0);
  return L;
}

// Assign the buffer pointers of c->dp from the layout (c->buf allocated).
void assign_buffers(fdlb_ctx* c, const Layout& L) {
  fdlb::DevParams& p = c->dp;
  char* b = (char*)c->buf;
  if (c->precision == FDLB_MIXED) {
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) c->pair[i][j] = (float*)(b + (2 * i + j) * L.arr);
    p.r3l = (float*)(b + 4 * L.arr);
    p.a4l = (float*)(b + 5 * L.arr);
    p.afl = (float*)(b + 6 * L.arr);
    p.dm = (float*)(b + 7 * L.arr);
    p.fa = (float*)(b + 8 * L.arr);
    p.fb = (float*)(b + 9 * L.arr);
    p.fc = (float*)(b + 10 * L.arr);
    p.mhi = (double*)(b + L.mhi);
    c->parity = 0;
    set_pair_pointers(c);
  } else {
    p.F = b + 0 * L.arr;
    p.F2 = b + 1 * L.arr;
    p.F3 = b + 2 * L.arr;
    p.A4 = b + 3 * L.arr;
    p.Af = b + 4 * L.arr;
    p.D = b + 5 * L.arr;
  }
  c->mom = (double*)(b + L.mom);
  p.status = (unsigned*)(b + L.mom + 4 * (size_t)p.N * sizeof(double));
}

// A binary64 scratch array of P * N values for moving a FDLB_MIXED state to
// or from the host: r3l and a4l, which hold nothing between steps.
double* mixed_exchange_buffer(fdlb_ctx* c) { return (double*)c->dp.r3l; }

int ensure_prepared(fdlb_ctx* c) {
  if (c->prepared) return FDLB_OK;
  cudaError_t me = cudaMemsetAsync(c->dp.status, 0, sizeof(unsigned), c->stream);
  if (me == cudaSuccess && c->batch)
    me = cudaMemsetAsync(c->dp.pstatus, 0, c->probs.size() * sizeof(unsigned), c->stream);
  if (me != cudaSuccess) return cuda_err(c, me, "status reset");
  int e = launch_stage_any(c, fdlb::kPrep, c->stream);
  if (e) return cuda_err(c, (cudaError_t)e, "prepare kernel launch");
  c->prepared = true;
  return FDLB_OK;
}

}  // namespace

namespace fdlb {

// Constants of a DevParams (lattice, grid, stage coefficients; the buffer
// pointers are left alone) for the arguments of fdlb_create, with the same
// checks.  Used by the allocation-free entry point (fdlb_noalloc.cu).
int params_for(const fdlb_grid* grid, int Qphi, int Qchi, double gamma, double tau, double dt,
               const fdlb_tableau* tableau, DevParams* out) {
  if (!grid || !out) return set_err(nullptr, FDLB_EINVAL, "grid or params is NULL");
  const fdlb_grid& g = *grid;
  if (g.d != 1 && g.d != 2) return set_err(nullptr, FDLB_EINVAL, "d must be 1 or 2 (got %d)", g.d);
  const int64_t ny = (g.d == 2) ? g.ny : 1;
  if (g.nx < 1 || ny < 1 || g.nx > (1 << 30) || ny > (1 << 30))
    return set_err(nullptr, FDLB_EINVAL, "bad cell counts nx=%lld ny=%lld", (long long)g.nx,
                   (long long)g.ny);
  // the kernels index cells with 32-bit offsets
  if (g.nx * ny >= ((int64_t)1 << 31))
    return set_err(nullptr, FDLB_EINVAL, "nx*ny = %lld cells: at most 2^31 - 1",
                   (long long)(g.nx * ny));
  if (!(g.x1 > g.x0) || (g.d == 2 && !(g.y1 > g.y0)))
    return set_err(nullptr, FDLB_EINVAL, "empty domain");
  if (g.bc != FDLB_BC_OUTLET && g.bc != FDLB_BC_PERIODIC)
    return set_err(nullptr, FDLB_EINVAL, "bc must be 0 (outlet) or 1 (periodic)");
  if (!supported_lattice(g.d, Qphi, Qchi))
    return set_err(nullptr, FDLB_EINVAL, "lattice d=%d Qphi=%d Qchi=%d not compiled", g.d, Qphi,
                   Qchi);
  if (!(gamma > 1.0) || !std::isfinite(gamma))
    return set_err(nullptr, FDLB_EINVAL, "gamma must be > 1");
  const double DK = 2.0 / (gamma - 1.0);
  if (DK - g.d < 0.0)
    return set_err(nullptr, FDLB_EINVAL, "gamma=%g gives D+K-d=%g < 0", gamma, DK - g.d);
  if (!(tau > 0.0) || !(dt > 0.0) || !std::isfinite(tau) || !std::isfinite(dt))
    return set_err(nullptr, FDLB_EINVAL, "tau and dt must be positive");
  fdlb_tableau tab;
  if (tableau) tab = *tableau;
  else paper_tableau(&tab);
  DevParams& p = *out;
  p.d = g.d;
  p.nx = (int)g.nx;
  p.ny = (int)ny;
  p.bc = g.bc;
  p.Qp = Qphi;
  p.Qc = Qchi;
  p.nphi = g.d == 1 ? Qphi : Qphi * Qphi;
  p.nchi = g.d == 1 ? Qchi : Qchi * Qchi;
  p.P = p.nphi + p.nchi;
  p.N = g.nx * ny;
  p.DK = DK;
  p.kchi = DK - g.d;
  const double dx = (g.x1 - g.x0) / (double)g.nx;
  const double dy = (g.d == 2) ? (g.y1 - g.y0) / (double)ny : 1.0;
  p.dtdx = dt / dx;
  p.dtdy = (g.d == 2) ? dt / dy : 0.0;
  double wp[kMaxQ], wc[kMaxQ];
  if (!gauss_hermite(Qphi, p.pp, wp) || !gauss_hermite(Qchi, p.pc, wc))
    return set_err(nullptr, FDLB_EINVAL, "Gauss-Hermite rule failed to converge");
  weighted_hermite_table(Qphi, p.pp, wp, p.wHp);
  weighted_hermite_table(Qchi, p.pc, wc, p.wHc);
  for (int i = 0; i < kMaxQ * kMaxQ; ++i) {
    split_float(p.wHp[i], &p.wHph[i], &p.wHpl[i]);
    split_float(p.wHc[i], &p.wHch[i], &p.wHcl[i]);
  }
  const double pmax = std::fmax(std::fabs(p.pp[Qphi - 1]), std::fabs(p.pc[Qchi - 1]));
  const double cfl = pmax * std::fmax(p.dtdx, p.dtdy);
  if (cfl > 1.0) return set_err(nullptr, FDLB_ECFL, "CFL = %g > 1", cfl);
  p.invDK = 1.0 / DK;
  for (int pop = 0; pop < p.P; ++pop) {
    double ax, ay;
    if (pop < p.nphi) {
      ax = p.pp[g.d == 1 ? pop : pop % Qphi];
      ay = g.d == 1 ? 0.0 : p.pp[pop / Qphi];
      p.p2[pop] = ax * ax + ay * ay;
    } else {
      const int q = pop - p.nphi;
      ax = p.pc[g.d == 1 ? q : q % Qchi];
      ay = g.d == 1 ? 0.0 : p.pc[q / Qchi];
      p.p2[pop] = 0.0;
    }
    p.px[pop] = ax;
    p.py[pop] = ay;
    p.cx[pop] = p.dtdx * ax;
    p.cy[pop] = p.dtdy * ay;
    split_float(ax, &p.pxh[pop], &p.pxl[pop]);
    split_float(ay, &p.pyh[pop], &p.pyl[pop]);
    split_float(p.p2[pop], &p.p2h[pop], &p.p2l[pop]);
  }
  const char* why = nullptr;
  if (!stage_coefficients(tab, dt / tau, &p.sc, &why))
    return set_err(nullptr, FDLB_EINVAL, "unsupported tableau: %s", why);
  return FDLB_OK;
}

// Record a context-less error for fdlb_last_error(NULL).
int record_error(int code, const char* msg) { return set_err(nullptr, code, "%s", msg); }

// Error recording, preparation and stage launch for the other host files.
int ctx_error(fdlb_ctx* c, int code, const char* msg) { return set_err(c, code, "%s", msg); }
int ctx_prepare(fdlb_ctx* c) { return ensure_prepared(c); }
int ctx_launch_stage(fdlb_ctx* c, int stage, cudaStream_t s) { return launch_stage_any(c, stage, s); }

}  // namespace fdlb

extern "C" {

int fdlb_named_tableau(int which, fdlb_tableau* out) {
  if (!out) return set_err(nullptr, FDLB_EINVAL, "out is NULL");
  if (which == FDLB_TABLEAU_IMEX_SSP3_433) paper_tableau(out);
  else if (which == FDLB_TABLEAU_EXPLICIT_SSPRK3) explicit_ssprk3_tableau(out);
  else return set_err(nullptr, FDLB_EINVAL, "unknown tableau %d", which);
  return FDLB_OK;
}

int fdlb_create(const fdlb_grid* grid, int Qphi, int Qchi, double gamma, double tau, double dt,
                const fdlb_tableau* tableau, int precision, void* cuda_stream, fdlb_ctx** out) {
  if (!out) return set_err(nullptr, FDLB_EINVAL, "out is NULL");
  *out = nullptr;
  if (!grid) return set_err(nullptr, FDLB_EINVAL, "grid is NULL");
  const fdlb_grid& g = *grid;
  if (g.d != 1 && g.d != 2) return set_err(nullptr, FDLB_EINVAL, "d must be 1 or 2 (got %d)", g.d);
  const int64_t ny = (g.d == 2) ? g.ny : 1;
  if (g.nx < 1 || ny < 1 || g.nx > (1 << 30) || ny > (1 << 30))
    return set_err(nullptr, FDLB_EINVAL, "bad cell counts nx=%lld ny=%lld", (long long)g.nx,
                   (long long)g.ny);
  // the kernels index cells with 32-bit offsets
  if (g.nx * ny >= ((int64_t)1 << 31))
    return set_err(nullptr, FDLB_EINVAL, "nx*ny = %lld cells: at most 2^31 - 1",
                   (long long)(g.nx * ny));
  if (!(g.x1 > g.x0) || (g.d == 2 && !(g.y1 > g.y0)))
    return set_err(nullptr, FDLB_EINVAL, "empty domain");
  if (g.bc != FDLB_BC_OUTLET && g.bc != FDLB_BC_PERIODIC)
    return set_err(nullptr, FDLB_EINVAL, "bc must be 0 (outlet) or 1 (periodic)");
  if (precision != FDLB_FP64 && precision != FDLB_MIXED)
    return set_err(nullptr, FDLB_EINVAL, "precision must be FDLB_FP64 or FDLB_MIXED (got %d)",
                   precision);
  if (!fdlb::supported_lattice(g.d, Qphi, Qchi))
    return set_err(nullptr, FDLB_EINVAL, "lattice d=%d Qphi=%d Qchi=%d not compiled", g.d, Qphi,
                   Qchi);
  if (!(gamma > 1.0) || !std::isfinite(gamma))
    return set_err(nullptr, FDLB_EINVAL, "gamma must be > 1");
  const double DK = 2.0 / (gamma - 1.0);
  if (DK - g.d < 0.0)
    return set_err(nullptr, FDLB_EINVAL, "gamma=%g gives D+K-d=%g < 0", gamma, DK - g.d);
  if (!(tau > 0.0) || !(dt > 0.0) || !std::isfinite(tau) || !std::isfinite(dt))
    return set_err(nullptr, FDLB_EINVAL, "tau and dt must be positive");
  const int64_t N = g.nx * ny;
  if (N > ((int64_t)1 << 31) / 2) return set_err(nullptr, FDLB_EINVAL, "too many cells");

  fdlb_tableau tab;
  if (tableau) tab = *tableau;
  else paper_tableau(&tab);

  fdlb_ctx* c = new (std::nothrow) fdlb_ctx();
  if (!c) return set_err(nullptr, FDLB_ENOMEM, "host allocation failed");
  c->grid = g;
  c->grid.ny = ny;
  c->custom_tableau = tableau != nullptr;
  c->gamma = gamma;
  c->tau = tau;
  c->dt = dt;
  c->precision = precision;
  c->stream = (cudaStream_t)cuda_stream;
  DevParams& p = c->dp;
  p.d = g.d;
  p.nx = (int)g.nx;
  p.ny = (int)ny;
  p.bc = g.bc;
  p.Qp = Qphi;
  p.Qc = Qchi;
  p.nphi = g.d == 1 ? Qphi : Qphi * Qphi;
  p.nchi = g.d == 1 ? Qchi : Qchi * Qchi;
  p.P = p.nphi + p.nchi;
  p.N = N;
  p.DK = DK;
  p.kchi = DK - g.d;
  const double dx = (g.x1 - g.x0) / (double)g.nx;
  const double dy = (g.d == 2) ? (g.y1 - g.y0) / (double)ny : 1.0;
  p.dtdx = dt / dx;
  p.dtdy = (g.d == 2) ? dt / dy : 0.0;
  double wp[kMaxQ], wc[kMaxQ];
  if (!gauss_hermite(Qphi, p.pp, wp) || !gauss_hermite(Qchi, p.pc, wc)) {
    delete c;
    return set_err(nullptr, FDLB_EINVAL, "Gauss-Hermite rule failed to converge");
  }
  weighted_hermite_table(Qphi, p.pp, wp, p.wHp);
  weighted_hermite_table(Qchi, p.pc, wc, p.wHc);
  for (int i = 0; i < kMaxQ * kMaxQ; ++i) {
    split_float(p.wHp[i], &p.wHph[i], &p.wHpl[i]);
    split_float(p.wHc[i], &p.wHch[i], &p.wHcl[i]);
  }
  // CFL condition |p| dt / ds <= 1 for all momenta (Sec. IV)
  const double pmax = std::fmax(std::fabs(p.pp[Qphi - 1]), std::fabs(p.pc[Qchi - 1]));
  const double cfl = pmax * std::fmax(p.dtdx, p.dtdy);
  if (cfl > 1.0) {
    delete c;
    return set_err(nullptr, FDLB_ECFL, "CFL = %g > 1", cfl);
  }
  p.invDK = 1.0 / DK;
  for (int pop = 0; pop < p.P; ++pop) {
    double ax, ay;
    if (pop < p.nphi) {
      ax = p.pp[g.d == 1 ? pop : pop % Qphi];
      ay = g.d == 1 ? 0.0 : p.pp[pop / Qphi];
      p.p2[pop] = ax * ax + ay * ay;
    } else {
      const int q = pop - p.nphi;
      ax = p.pc[g.d == 1 ? q : q % Qchi];
      ay = g.d == 1 ? 0.0 : p.pc[q / Qchi];
      p.p2[pop] = 0.0;
    }
    p.px[pop] = ax;
    p.py[pop] = ay;
    p.cx[pop] = p.dtdx * ax;
    p.cy[pop] = p.dtdy * ay;
    split_float(ax, &p.pxh[pop], &p.pxl[pop]);
    split_float(ay, &p.pyh[pop], &p.pyl[pop]);
    split_float(p.p2[pop], &p.p2h[pop], &p.p2l[pop]);
  }
  const char* why = nullptr;
  if (!stage_coefficients(tab, dt / tau, &p.sc, &why)) {
    delete c;
    return set_err(nullptr, FDLB_EINVAL, "unsupported tableau: %s", why);
  }
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_err(nullptr, e, "cudaGetDevice");
  }
  p.precision = precision;
  const Layout lay = buffer_layout(precision, p.P, N);
  c->buf_bytes = lay.total;
  e = cudaMalloc(&c->buf, c->buf_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    const size_t want = c->buf_bytes;
    delete c;
    return set_err(nullptr, FDLB_ENOMEM, "cudaMalloc(%zu) failed: %s", want,
                   cudaGetErrorString(e));
  }
  assign_buffers(c, lay);
  e = cudaMallocHost(&c->status_host, sizeof(unsigned));
  if (e == cudaSuccess && precision == FDLB_MIXED) e = (cudaError_t)fdlb::mixed_setup(p);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->buf, 0, c->buf_bytes, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    int rc = cuda_err(nullptr, e, "context set-up");
    fdlb_destroy(c);
    return rc;
  }
  *out = c;
  return FDLB_OK;
}

int fdlb_init_riemann(fdlb_ctx* c, const double* states, int nq, double xsplit, double ysplit) {
  if (!c) return set_err(nullptr, FDLB_EINVAL, "ctx is NULL");
  if (c->batch) return set_err(c, FDLB_EINVAL, "batch context: use fdlb_batch_init_riemann");
  if (!states) return set_err(c, FDLB_EINVAL, "states is NULL");
  if (!std::isfinite(xsplit) || !std::isfinite(ysplit))
    return set_err(c, FDLB_EINVAL, "non-finite membrane position");
  const int d = c->dp.d;
  if ((d == 1 && nq != 2) || (d == 2 && nq != 4))
    return set_err(c, FDLB_EINVAL, "nq must be 2 in 1-D and 4 in 2-D");
  const int w = d + 2;
  for (int q = 0; q < nq; ++q) {
    const double rho = states[q * w], P = states[q * w + w - 1];
    for (int j = 0; j < w; ++j)
      if (!std::isfinite(states[q * w + j])) return set_err(c, FDLB_EINVAL, "non-finite state");
    if (!(rho > 0.0) || !(P > 0.0)) return set_err(c, FDLB_EINVAL, "rho and P must be > 0");
  }
  const fdlb_grid& g = c->grid;
  const double sx = fdlb::split_in_cells(xsplit, g.x0, g.x1, g.nx);
  const double sy = (d == 2) ? fdlb::split_in_cells(ysplit, g.y0, g.y1, g.ny) : 0.0;
  int e = fdlb::launch_init_riemann(c->dp, states, nq, sx, sy, c->stream);
  if (e) return cuda_err(c, (cudaError_t)e, "init kernel launch");
  c->prepared = false;
  return ensure_prepared(c);
}

int fdlb_step(fdlb_ctx* c, int64_t nsteps) {
  if (!c) return set_err(nullptr, FDLB_EINVAL, "ctx is NULL");
  if (nsteps < 0) return set_err(c, FDLB_EINVAL, "nsteps < 0");
  int rc = ensure_prepared(c);
  if (rc) return rc;
  int64_t left = nsteps;
  if (nsteps >= kGraphSteps) {
    rc = ensure_graph(c);
    if (rc) return rc;
    for (; left >= kGraphSteps; left -= kGraphSteps) {
      cudaError_t ge = cudaGraphLaunch(c->graph_exec[c->parity], c->stream);
      if (ge != cudaSuccess) return cuda_err(c, ge, "cudaGraphLaunch");
    }
  }
  for (int64_t s = 0; s < left; ++s) {
    for (int st : {fdlb::kStage3, fdlb::kStage4, fdlb::kFinal}) {
      int e = step_launch(c, st, c->stream);
      if (e) return cuda_err(c, (cudaError_t)e, "stage kernel launch");
    }
  }
  cudaError_t e = cudaMemcpyAsync(c->status_host, c->dp.status, sizeof(unsigned),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "fdlb_step");
  if (*c->status_host & 1u)
    return set_err(c, FDLB_EUNSTABLE, "a cell reached n <= 0, T <= 0 or a non-finite moment");
  return FDLB_OK;
}

int fdlb_step_timed(fdlb_ctx* c, int64_t nsteps, double* stage_ms) {
  if (!c) return set_err(nullptr, FDLB_EINVAL, "ctx is NULL");
  if (nsteps < 0 || !stage_ms) return set_err(c, FDLB_EINVAL, "bad nsteps or stage_ms");
  for (int i = 0; i < 3; ++i) stage_ms[i] = 0.0;
  int rc = ensure_prepared(c);
  if (rc) return rc;
  const int kinds[3] = {fdlb::kStage3, fdlb::kStage4, fdlb::kFinal};
  const size_t nev = (size_t)(3 * nsteps + 1);
  std::vector<cudaEvent_t> ev(nev, nullptr);
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < nev && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], c->stream);
  for (int64_t s = 0; s < nsteps && e == cudaSuccess; ++s) {
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
      int le = step_launch(c, kinds[k], c->stream);
      if (le) e = (cudaError_t)le;
      if (e == cudaSuccess) e = cudaEventRecord(ev[3 * s + k + 1], c->stream);
    }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->status_host, c->dp.status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                        c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  for (int64_t s = 0; s < nsteps && e == cudaSuccess; ++s)
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
      float ms = 0.0f;
      e = cudaEventElapsedTime(&ms, ev[3 * s + k], ev[3 * s + k + 1]);
      stage_ms[k] += ms;
    }
  for (size_t i = 0; i < nev; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess) return cuda_err(c, e, "fdlb_step_timed");
  if (*c->status_host & 1u)
    return set_err(c, FDLB_EUNSTABLE, "a cell reached n <= 0, T <= 0 or a non-finite moment");
  return FDLB_OK;
}

int fdlb_moments(fdlb_ctx* c, double* n, double* ux, double* uy, double* T, int on_device) {
  if (!c) return set_err(nullptr, FDLB_EINVAL, "ctx is NULL");
  if (!n || !ux || !T || (c->dp.d == 2 && !uy))
    return set_err(c, FDLB_EINVAL, "NULL output pointer");
  const int64_t N = c->dp.N;
  if (on_device) {
    int e = fdlb::launch_moments(c->dp, n, ux, c->dp.d == 2 ? uy : nullptr, T, c->stream);
    if (e) return cuda_err(c, (cudaError_t)e, "moments kernel launch");
    return FDLB_OK;
  }
  double* tmp = c->mom;
  int le = fdlb::launch_moments(c->dp, tmp, tmp + N, c->dp.d == 2 ? tmp + 2 * N : nullptr,
                                tmp + 3 * N, c->stream);
  if (le) return cuda_err(c, (cudaError_t)le, "moments kernel launch");
  double* dst[4] = {n, ux, c->dp.d == 2 ? uy : nullptr, T};
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 4 && e == cudaSuccess; ++i)
    if (dst[i])
      e = cudaMemcpyAsync(dst[i], tmp + i * N, N * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "fdlb_moments copy");
  return FDLB_OK;
}

int fdlb_moments_adjoint(fdlb_ctx* c, const double* nbar, const double* uxbar,
                         const double* uybar, const double* Tbar, double* Fbar) {
  if (!c) return set_err(nullptr, FDLB_EINVAL, "ctx is NULL");
  if (!Fbar) return set_err(c, FDLB_EINVAL, "Fbar is NULL");
  if (c->batch || c->precision != FDLB_FP64)
    return set_err(c, FDLB_EINVAL, "fdlb_moments_adjoint: single-problem binary64 contexts");
  int e = fdlb::launch_moments_adjoint(c->dp, nbar, uxbar, c->dp.d == 2 ? uybar : nullptr, Tbar,
                                       Fbar, c->stream);
  if (e) return cuda_err(c, (cudaError_t)e, "moments adjoint kernel launch");
  return FDLB_OK;
}

size_t fdlb_state_bytes(const fdlb_ctx* c) {
  if (!c) return 0;
  return (size_t)c->dp.P * (size_t)c->dp.N * sizeof(double);
}

int fdlb_get_state(fdlb_ctx* c, void* dst, int on_device) {
  if (!c) return set_err(nullptr, FDLB_EINVAL, "ctx is NULL");
  if (!dst) return set_err(c, FDLB_EINVAL, "dst is NULL");
  cudaError_t e = cudaSuccess;
  if (c->precision == FDLB_MIXED) {
    // the exact binary64 value hi + lo of every population
    double* dev = on_device ? (double*)dst : mixed_exchange_buffer(c);
    const int64_t n = (int64_t)c->dp.P * c->dp.N;
    int le = fdlb::launch_pair_to_double(c->dp.sh, c->dp.sl, dev, n, c->stream);
    if (le) e = (cudaError_t)le;
    if (e == cudaSuccess && !on_device)
      e = cudaMemcpyAsync(dst, dev, fdlb_state_bytes(c), cudaMemcpyDeviceToHost, c->stream);
  } else {
    e = cudaMemcpyAsync(dst, c->dp.F, fdlb_state_bytes(c),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
  }
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "fdlb_get_state");
  return FDLB_OK;
}

int fdlb_set_state(fdlb_ctx* c, const void* src, int on_device) {
  if (!c) return set_err(nullptr, FDLB_EINVAL, "ctx is NULL");
  if (!src) return set_err(c, FDLB_EINVAL, "src is NULL");
  cudaError_t e = cudaSuccess;
  if (c->precision == FDLB_MIXED) {
    // each binary64 value v becomes hi = v rounded, lo = (v - hi) rounded
    const double* dev = (const double*)src;
    if (!on_device) {
      e = cudaMemcpyAsync(mixed_exchange_buffer(c), src, fdlb_state_bytes(c),
                          cudaMemcpyHostToDevice, c->stream);
      dev = mixed_exchange_buffer(c);
    }
    const int64_t n = (int64_t)c->dp.P * c->dp.N;
    if (e == cudaSuccess) {
      int le = fdlb::launch_double_to_pair(dev, c->dp.sh, c->dp.sl, n, c->stream);
      if (le) e = (cudaError_t)le;
    }
  } else {
    e = cudaMemcpyAsync(c->dp.F, src, fdlb_state_bytes(c),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
  }
  if (e != cudaSuccess) return cuda_err(c, e, "fdlb_set_state");
  c->prepared = false;
  int rc = ensure_prepared(c);
  if (rc) return rc;
  if (!on_device) {
    // the source may be pageable memory the caller frees right after
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "fdlb_set_state");
  }
  return FDLB_OK;
}

// ---- batches of 1-D problems -------------------------------------------------

namespace {

int upload_work(fdlb_ctx* c) {
  const int tx = fdlb::batch_tile_cells(c->dp.variant);
  std::vector<fdlb::WorkItem> work;
  for (int i = 0; i < (int)c->probs.size(); ++i)
    for (int x = 0; x < c->probs[i].nx; x += tx) work.push_back(fdlb::WorkItem{i, x});
  if (c->work_dev) cudaFree(c->work_dev);
  c->work_dev = nullptr;
  cudaError_t e = cudaMalloc(&c->work_dev, work.size() * sizeof(fdlb::WorkItem));
  if (e != cudaSuccess) return set_err(c, FDLB_ENOMEM, "work list: %s", cudaGetErrorString(e));
  e = cudaMemcpyAsync(c->work_dev, work.data(), work.size() * sizeof(fdlb::WorkItem),
                      cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "work list upload");
  c->dp.work = c->work_dev;
  c->dp.nwork = (int)work.size();
  return FDLB_OK;
}

int upload_probs(fdlb_ctx* c) {
  cudaError_t e = cudaMemcpyAsync(c->probs_dev, c->probs.data(),
                                  c->probs.size() * sizeof(fdlb::BatchProblem),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "problem table upload");
  return FDLB_OK;
}

}  // namespace

int fdlb_create_batch(int nprob, const int64_t* nx, const double* gamma, double x0, double x1,
                      int Qphi, int Qchi, double tau, double dt, int precision, void* cuda_stream,
                      fdlb_ctx** out) {
  if (!out) return set_err(nullptr, FDLB_EINVAL, "out is NULL");
  *out = nullptr;
  if (nprob < 1 || !nx || !gamma) return set_err(nullptr, FDLB_EINVAL, "nprob < 1 or NULL arrays");
  if (!(x1 > x0)) return set_err(nullptr, FDLB_EINVAL, "empty domain");
  if (precision != FDLB_FP64 && precision != FDLB_MIXED)
    return set_err(nullptr, FDLB_EINVAL, "precision must be FDLB_FP64 or FDLB_MIXED");
  if (!((Qphi == 8 && Qchi == 8) || (Qphi == 5 && Qchi == 3)))
    return set_err(nullptr, FDLB_EINVAL, "batch lattice Qphi=%d Qchi=%d not compiled", Qphi, Qchi);
  if (!(tau > 0.0) || !(dt > 0.0)) return set_err(nullptr, FDLB_EINVAL, "tau and dt must be positive");
  // lattice, coefficients and tables of the first problem; gas constants per problem
  fdlb_grid g{1, nx[0], 1, x0, x1, 0.0, 1.0, FDLB_BC_OUTLET};
  fdlb::DevParams tmpl{};
  int rc = fdlb::params_for(&g, Qphi, Qchi, gamma[0], tau, dt, nullptr, &tmpl);
  if (rc) return rc;
  const double pmax = std::fmax(std::fabs(tmpl.pp[Qphi - 1]), std::fabs(tmpl.pc[Qchi - 1]));
  std::vector<fdlb::BatchProblem> probs(nprob);
  int64_t total = 0;
  for (int i = 0; i < nprob; ++i) {
    if (nx[i] < 1 || nx[i] > (1 << 28)) return set_err(nullptr, FDLB_EINVAL, "problem %d: bad nx", i);
    const double gm = gamma[i];
    if (!(gm > 1.0) || !std::isfinite(gm)) return set_err(nullptr, FDLB_EINVAL, "problem %d: gamma", i);
    const double DK = 2.0 / (gm - 1.0);
    if (DK - 1.0 < 0.0) return set_err(nullptr, FDLB_EINVAL, "problem %d: D+K-d < 0", i);
    const double dx = (x1 - x0) / (double)nx[i];
    if (pmax * dt / dx > 1.0)
      return set_err(nullptr, FDLB_ECFL, "problem %d: CFL = %g > 1", i, pmax * dt / dx);
    fdlb::BatchProblem& b = probs[i];
    b = fdlb::BatchProblem{};
    b.base = total;
    b.nx = (int)nx[i];
    b.kchi = DK - 1.0;
    b.invDK = 1.0 / DK;
    b.dtdx = dt / dx;
    b.x0 = x0;
    b.x1 = x1;
    b.split = fdlb::split_in_cells(0.5 * (x0 + x1), x0, x1, nx[i]);
    total += nx[i];
    // the kernels index cells with 32-bit offsets
    if (total >= ((int64_t)1 << 31))
      return set_err(nullptr, FDLB_EINVAL, "batch of more than 2^31 - 1 cells");
  }
  if (total > ((int64_t)1 << 31) / 2) return set_err(nullptr, FDLB_EINVAL, "too many cells");
  fdlb_ctx* c = new (std::nothrow) fdlb_ctx();
  if (!c) return set_err(nullptr, FDLB_ENOMEM, "host allocation failed");
  c->batch = true;
  c->probs = probs;
  c->stream = (cudaStream_t)cuda_stream;
  c->precision = precision;
  c->tau = tau;
  c->dt = dt;
  c->grid = fdlb_grid{1, total, 1, x0, x1, 0.0, 1.0, FDLB_BC_OUTLET};
  fdlb::DevParams& p = c->dp;
  p = tmpl;
  p.nx = (int)total;  // not used by the batch kernels (per-problem sizes)
  p.N = total;
  p.precision = precision;
  p.nprob = nprob;
  p.variant = 0;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_err(nullptr, e, "device query");
  }
  p.bgrid = 4 * c->nsm;
  const size_t pstat_bytes = ((size_t)nprob * sizeof(unsigned) + 255) / 256 * 256;
  const Layout lay = buffer_layout(precision, p.P, total);
  c->buf_bytes = lay.total + pstat_bytes;
  e = cudaMalloc(&c->buf, c->buf_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->probs_dev, nprob * sizeof(fdlb::BatchProblem));
  if (e != cudaSuccess) {
    cudaGetLastError();
    fdlb_destroy(c);
    return set_err(nullptr, FDLB_ENOMEM, "batch allocation failed: %s", cudaGetErrorString(e));
  }
  assign_buffers(c, lay);
  p.pstatus = (unsigned*)((char*)c->buf + lay.total);
  p.probs = c->probs_dev;
  e = cudaMallocHost(&c->status_host, sizeof(unsigned));
  if (e == cudaSuccess && precision == FDLB_MIXED) e = (cudaError_t)fdlb::mixed_setup(p);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->buf, 0, c->buf_bytes, c->stream);
  if (e != cudaSuccess) {
    int r = cuda_err(nullptr, e, "batch set-up");
    fdlb_destroy(c);
    return r;
  }
  if ((rc = upload_probs(c)) || (rc = upload_work(c))) {
    std::string msg = c->err;
    fdlb_destroy(c);
    return set_err(nullptr, rc, "%s", msg.c_str());
  }
  *out = c;
  return FDLB_OK;
}

int fdlb_batch_init_riemann(fdlb_ctx* c, const double* states, const double* xsplit) {
  if (!c) return set_err(nullptr, FDLB_EINVAL, "ctx is NULL");
  if (!c->batch) return set_err(c, FDLB_EINVAL, "not a batch context");
  if (!states) return set_err(c, FDLB_EINVAL, "states is NULL");
  for (size_t i = 0; i < c->probs.size(); ++i) {
    for (int q = 0; q < 2; ++q) {
      const double* st = states + 6 * i + 3 * q;
      if (!std::isfinite(st[0]) || !std::isfinite(st[1]) || !std::isfinite(st[2]) ||
          !(st[0] > 0.0) || !(st[2] > 0.0))
        return set_err(c, FDLB_EINVAL, "problem %zu: rho and P must be finite and > 0", i);
      for (int j = 0; j < 3; ++j) c->probs[i].st[q][j] = st[j];
    }
    if (xsplit) {
      if (!std::isfinite(xsplit[i])) return set_err(c, FDLB_EINVAL, "problem %zu: non-finite xsplit", i);
      fdlb::BatchProblem& b = c->probs[i];
      b.split = fdlb::split_in_cells(xsplit[i], b.x0, b.x1, b.nx);
    }
  }
  int rc = upload_probs(c);
  if (rc) return rc;
  int e = fdlb::launch_batch_init(c->dp, c->stream);
  if (e) return cuda_err(c, (cudaError_t)e, "batch init kernel launch");
  c->prepared = false;
  return ensure_prepared(c);
}

int fdlb_batch_status(fdlb_ctx* c, unsigned* flags) {
  if (!c || !c->batch || !flags) return set_err(c, FDLB_EINVAL, "not a batch context or NULL");
  cudaError_t e = cudaMemcpyAsync(flags, c->dp.pstatus, c->probs.size() * sizeof(unsigned),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "fdlb_batch_status");
  return FDLB_OK;
}

int fdlb_batch_offsets(const fdlb_ctx* c, int64_t* base) {
  if (!c || !c->batch || !base) return set_err(nullptr, FDLB_EINVAL, "not a batch context");
  for (size_t i = 0; i < c->probs.size(); ++i) base[i] = c->probs[i].base;
  return FDLB_OK;
}

int fdlb_autotune(fdlb_ctx* c, int trial_steps, int* variant_out, int* ctas_per_sm_out) {
  if (!c) return set_err(nullptr, FDLB_EINVAL, "ctx is NULL");
  if (!c->batch) return set_err(c, FDLB_EINVAL, "autotuning applies to batch contexts");
  if (trial_steps < 1) trial_steps = 2;
  int rc = ensure_prepared(c);
  if (rc) return rc;
  // keep the state (as binary64 values): every trial starts from it
  const size_t bytes = fdlb_state_bytes(c);
  void* saved = nullptr;
  cudaError_t e = cudaMalloc(&saved, bytes);
  if (e != cudaSuccess) return set_err(c, FDLB_ENOMEM, "autotune buffer: %s", cudaGetErrorString(e));
  auto put_state = [&](bool restore) -> cudaError_t {
    if (c->precision == FDLB_MIXED) {
      const int64_t n = (int64_t)c->dp.P * c->dp.N;
      return (cudaError_t)(restore ? fdlb::launch_double_to_pair((const double*)saved, c->dp.sh,
                                                                 c->dp.sl, n, c->stream)
                                   : fdlb::launch_pair_to_double(c->dp.sh, c->dp.sl,
                                                                 (double*)saved, n, c->stream));
    }
    return restore ? cudaMemcpyAsync(c->dp.F, saved, bytes, cudaMemcpyDeviceToDevice, c->stream)
                   : cudaMemcpyAsync(saved, c->dp.F, bytes, cudaMemcpyDeviceToDevice, c->stream);
  };
  e = put_state(false);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  const int ctas[] = {2, 4, 8, 16};
  float best = 1e30f;
  int best_v = 0, best_k = 4;
  for (int v = 0; v < fdlb::kBatchVariants && e == cudaSuccess && !rc; ++v) {
    c->dp.variant = v;
    if ((rc = upload_work(c))) break;
    for (int k : ctas) {
      c->dp.bgrid = k * c->nsm;
      e = put_state(true);
      int le = e == cudaSuccess ? launch_stage_any(c, fdlb::kPrep, c->stream) : 0;
      if (e == cudaSuccess) e = cudaEventRecord(t0, c->stream);
      for (int s = 0; s < trial_steps && e == cudaSuccess && !le; ++s)
        for (int st : {fdlb::kStage3, fdlb::kStage4, fdlb::kFinal})
          if (!le) le = step_launch(c, st, c->stream);
      if (le) e = (cudaError_t)le;
      if (e == cudaSuccess) e = cudaEventRecord(t1, c->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
      if (e == cudaSuccess && ms < best) {
        best = ms;
        best_v = v;
        best_k = k;
      }
    }
  }
  // restore the state and adopt the fastest shape
  if (e == cudaSuccess && !rc) {
    c->dp.variant = best_v;
    c->dp.bgrid = best_k * c->nsm;
    rc = upload_work(c);
    if (!rc) e = put_state(true);
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaStreamSynchronize(c->stream);
  cudaFree(saved);
  drop_graph(c);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_err(c, e, "fdlb_autotune");
  c->prepared = false;
  rc = ensure_prepared(c);
  if (rc) return rc;
  if (variant_out) *variant_out = best_v;
  if (ctas_per_sm_out) *ctas_per_sm_out = best_k;
  return FDLB_OK;
}

int fdlb_batch_set_tiling(fdlb_ctx* c, int variant, int ctas_per_sm) {
  if (!c || !c->batch) return set_err(c, FDLB_EINVAL, "not a batch context");
  if (variant < 0 || variant >= fdlb::kBatchVariants || ctas_per_sm < 1 || ctas_per_sm > 64)
    return set_err(c, FDLB_EINVAL, "variant in [0, %d), ctas_per_sm in [1, 64]", fdlb::kBatchVariants);
  c->dp.variant = variant;
  c->dp.bgrid = ctas_per_sm * c->nsm;
  drop_graph(c);
  return upload_work(c);
}

int fdlb_lattice_nodes(int Q, double* p, double* w) {
  if (!p || !w || Q < 1 || Q > kMaxQ) return set_err(nullptr, FDLB_EINVAL, "bad Q or NULL arrays");
  if (!gauss_hermite(Q, p, w)) return set_err(nullptr, FDLB_EINVAL, "Gauss-Hermite rule failed");
  return FDLB_OK;
}

int fdlb_npop(const fdlb_ctx* c) { return c ? c->dp.P : 0; }

int64_t fdlb_ncells(const fdlb_ctx* c) { return c ? c->dp.N : 0; }

int fdlb_set_stream(fdlb_ctx* c, void* stream) {
  if (!c) return set_err(nullptr, FDLB_EINVAL, "ctx is NULL");
  c->stream = (cudaStream_t)stream;
  return FDLB_OK;
}

int fdlb_launches_per_step(const fdlb_ctx* c) { return c ? 3 : 0; }

void fdlb_destroy(fdlb_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  drop_graph(c);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  if (c->probs_dev) cudaFree(c->probs_dev);
  if (c->work_dev) cudaFree(c->work_dev);
  if (c->buf) cudaFree(c->buf);
  if (c->adj_buf) cudaFree(c->adj_buf);
  if (c->status_host) cudaFreeHost(c->status_host);
  delete c;
}

const char* fdlb_last_error(const fdlb_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.empty() ? "no error" : c->err.c_str();
}

}  // extern "C"
