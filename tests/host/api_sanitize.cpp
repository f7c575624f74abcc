// Driver of the library's host code (csrc/fdlb_api.cpp) for the address and
// undefined-behaviour sanitizers, without a GPU: the kernel launchers of the
// .cu files are replaced by stand-ins that report "no device", and every
// entry point is called with the arguments it must reject and with valid
// ones (which then fail at the first CUDA call, as they do on a machine
// without a GPU).  The checks are the return codes; the sanitizers abort on
// any out-of-bounds access, leak or undefined operation in the host logic:
// the Gauss-Hermite rule, the tableau reduction, argument validation and
// error reporting.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "fdlb.h"
#include "fdlb_internal.h"

namespace fdlb {
bool supported_lattice(int d, int Qp, int Qc) {
  return (d == 1 || d == 2) && ((Qp == 8 && Qc == 8) || (Qp == 5 && Qc == 3) || (Qp == 3 && Qc == 3));
}
int launch_stage(const DevParams&, int, cudaStream_t) { return (int)cudaErrorNoDevice; }
int launch_init_riemann(const DevParams&, const double*, int, double, double, cudaStream_t) {
  return (int)cudaErrorNoDevice;
}
int launch_moments(const DevParams&, double*, double*, double*, double*, cudaStream_t) {
  return (int)cudaErrorNoDevice;
}
int launch_moments_adjoint(const DevParams&, const double*, const double*, const double*,
                           const double*, double*, cudaStream_t) {
  return (int)cudaErrorNoDevice;
}
int launch_batch_stage(const DevParams&, int, cudaStream_t) { return (int)cudaErrorNoDevice; }
int launch_batch_init(const DevParams&, cudaStream_t) { return (int)cudaErrorNoDevice; }
int batch_tile_cells(int) { return 127; }
int mixed_setup(const DevParams&) { return (int)cudaErrorNoDevice; }
int launch_pair_to_double(const float*, const float*, double*, int64_t, cudaStream_t) {
  return (int)cudaErrorNoDevice;
}
int launch_double_to_pair(const double*, float*, float*, int64_t, cudaStream_t) {
  return (int)cudaErrorNoDevice;
}
}  // namespace fdlb

static int fails = 0;
#define EXPECT(cond)                                                     \
  do {                                                                   \
    if (!(cond)) {                                                       \
      std::fprintf(stderr, "%s:%d: %s\n", __FILE__, __LINE__, #cond);   \
      ++fails;                                                           \
    }                                                                    \
  } while (0)

static int create(fdlb_grid g, int Qp, int Qc, double gamma, double tau, double dt,
                  const fdlb_tableau* t = nullptr, int prec = FDLB_FP64) {
  fdlb_ctx* c = reinterpret_cast<fdlb_ctx*>(1);
  const int rc = fdlb_create(&g, Qp, Qc, gamma, tau, dt, t, prec, nullptr, &c);
  if (rc == FDLB_OK) {  // a machine with a GPU: the set-up went through
    fdlb_destroy(c);
    return rc;
  }
  EXPECT(c == nullptr);  // no context on failure
  EXPECT(std::strlen(fdlb_last_error(nullptr)) > 0);
  return rc;
}

int main() {
  // Gauss-Hermite rules: every supported order, rejected orders
  double p[16], w[16];
  for (int Q = 1; Q <= 16; ++Q) {
    EXPECT(fdlb_lattice_nodes(Q, p, w) == FDLB_OK);
    double sw = 0.0;
    for (int k = 0; k < Q; ++k) sw += w[k];
    EXPECT(std::fabs(sw - 1.0) < 1e-13);
  }
  EXPECT(fdlb_lattice_nodes(0, p, w) == FDLB_EINVAL);
  EXPECT(fdlb_lattice_nodes(17, p, w) == FDLB_EINVAL);
  EXPECT(fdlb_lattice_nodes(8, nullptr, w) == FDLB_EINVAL);
  // named tableaux
  fdlb_tableau t;
  EXPECT(fdlb_named_tableau(FDLB_TABLEAU_IMEX_SSP3_433, &t) == FDLB_OK && t.r == 4);
  EXPECT(fdlb_named_tableau(FDLB_TABLEAU_EXPLICIT_SSPRK3, &t) == FDLB_OK && t.r == 4);
  EXPECT(fdlb_named_tableau(7, &t) == FDLB_EINVAL);
  EXPECT(fdlb_named_tableau(0, nullptr) == FDLB_EINVAL);

  const fdlb_grid g1{1, 400, 1, -0.5, 0.5, 0.0, 1.0, FDLB_BC_OUTLET};
  const fdlb_grid g2{2, 37, 29, 0.0, 1.0, 0.0, 1.0, FDLB_BC_PERIODIC};
  // rejected arguments
  fdlb_ctx* c = nullptr;
  EXPECT(fdlb_create(nullptr, 8, 8, 1.4, 1e-6, 5e-5, nullptr, FDLB_FP64, nullptr, &c) == FDLB_EINVAL);
  EXPECT(fdlb_create(&g1, 8, 8, 1.4, 1e-6, 5e-5, nullptr, FDLB_FP64, nullptr, nullptr) == FDLB_EINVAL);
  fdlb_grid b = g1;
  b.d = 3;
  EXPECT(create(b, 8, 8, 1.4, 1e-6, 5e-5) == FDLB_EINVAL);
  b = g1;
  b.nx = 0;
  EXPECT(create(b, 8, 8, 1.4, 1e-6, 5e-5) == FDLB_EINVAL);
  b = g2;
  b.nx = b.ny = 1 << 16;  // 2^32 cells
  EXPECT(create(b, 8, 8, 1.4, 1e-6, 1e-7) == FDLB_EINVAL);
  b = g1;
  b.x1 = b.x0;
  EXPECT(create(b, 8, 8, 1.4, 1e-6, 5e-5) == FDLB_EINVAL);
  b = g1;
  b.bc = 5;
  EXPECT(create(b, 8, 8, 1.4, 1e-6, 5e-5) == FDLB_EINVAL);
  EXPECT(create(g1, 8, 8, 1.4, 1e-6, 5e-5, nullptr, 9) == FDLB_EINVAL);
  EXPECT(create(g1, 7, 7, 1.4, 1e-6, 5e-5) == FDLB_EINVAL);
  EXPECT(create(g1, 8, 8, 1.0, 1e-6, 5e-5) == FDLB_EINVAL);
  EXPECT(create(g1, 8, 8, NAN, 1e-6, 5e-5) == FDLB_EINVAL);
  EXPECT(create(g2, 8, 8, 2.5, 1e-6, 5e-5) == FDLB_EINVAL);  // D + K - d < 0
  EXPECT(create(g1, 8, 8, 1.4, 0.0, 5e-5) == FDLB_EINVAL);
  EXPECT(create(g1, 8, 8, 1.4, 1e-6, -1.0) == FDLB_EINVAL);
  EXPECT(create(g1, 8, 8, 1.4, 1e-6, 1e-2) == FDLB_ECFL);
  fdlb_tableau bad;
  fdlb_named_tableau(FDLB_TABLEAU_IMEX_SSP3_433, &bad);
  bad.At[0 * 4 + 0] = 1.0;  // explicit diagonal
  EXPECT(create(g1, 8, 8, 1.4, 1e-6, 5e-5, &bad) == FDLB_EINVAL);
  bad.r = 3;
  EXPECT(create(g1, 8, 8, 1.4, 1e-6, 5e-5, &bad) == FDLB_EINVAL);
  // valid arguments: the context set-up reaches CUDA and reports its failure
  for (int prec : {FDLB_FP64, FDLB_MIXED}) {
    const int rc1 = create(g1, 8, 8, 1.4, 1e-6, 5e-5, nullptr, prec);
    const int rc2 = create(g2, 5, 3, 5.0 / 3.0, 1e-5, 5e-4, nullptr, prec);
    EXPECT(rc1 == FDLB_OK || rc1 == FDLB_ECUDA || rc1 == FDLB_ENOMEM);
    EXPECT(rc2 == FDLB_OK || rc2 == FDLB_ECUDA || rc2 == FDLB_ENOMEM);
  }
  // batches
  const int64_t nxs[3] = {256, 1000, 4096};
  const double gms[3] = {1.1, 1.4, 5.0 / 3.0};
  EXPECT(fdlb_create_batch(0, nxs, gms, -0.5, 0.5, 8, 8, 1e-6, 2e-5, FDLB_MIXED, nullptr, &c) ==
         FDLB_EINVAL);
  EXPECT(fdlb_create_batch(3, nxs, gms, -0.5, 0.5, 8, 8, 1e-6, 2e-5, 4, nullptr, &c) == FDLB_EINVAL);
  EXPECT(fdlb_create_batch(3, nxs, gms, -0.5, 0.5, 3, 3, 1e-6, 2e-5, FDLB_MIXED, nullptr, &c) ==
         FDLB_EINVAL);
  EXPECT(fdlb_create_batch(3, nxs, gms, -0.5, 0.5, 8, 8, 1e-6, 1e-3, FDLB_MIXED, nullptr, &c) ==
         FDLB_ECFL);
  const int rcb = fdlb_create_batch(3, nxs, gms, -0.5, 0.5, 8, 8, 1e-6, 2e-5, FDLB_MIXED, nullptr, &c);
  EXPECT(rcb == FDLB_ECUDA || rcb == FDLB_ENOMEM);
  // NULL contexts
  EXPECT(fdlb_step(nullptr, 1) == FDLB_EINVAL);
  EXPECT(fdlb_moments(nullptr, nullptr, nullptr, nullptr, nullptr, 0) == FDLB_EINVAL);
  EXPECT(fdlb_moments_adjoint(nullptr, nullptr, nullptr, nullptr, nullptr, nullptr) == FDLB_EINVAL);
  EXPECT(fdlb_get_state(nullptr, nullptr, 0) == FDLB_EINVAL);
  EXPECT(fdlb_set_state(nullptr, nullptr, 0) == FDLB_EINVAL);
  EXPECT(fdlb_init_riemann(nullptr, nullptr, 2, 0.0, 0.0) == FDLB_EINVAL);
  EXPECT(fdlb_state_bytes(nullptr) == 0 && fdlb_npop(nullptr) == 0 && fdlb_ncells(nullptr) == 0);
  fdlb_destroy(nullptr);
  EXPECT(std::strlen(fdlb_last_error(nullptr)) > 0);
  if (fails) std::fprintf(stderr, "%d failed expectations\n", fails);
  else std::printf("host API sanitize driver: ok\n");
  return fails ? 1 : 0;
}
