// fdlb_internal.h -- parameters shared by the host API (fdlb_api.cpp) and the
// sm_103a kernels (fdlb_kernels.cu).  Not part of the public C ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace fdlb {

constexpr int kMaxQ = 16;  // largest Gauss-Hermite order per axis
constexpr int kMaxPop = 128;  // largest population count of a compiled lattice (2-D, Q = 8)

// Coefficients of the fused IMEX stages.  With lam = dt/tau, e_i = lam/(1 +
// a_ii lam) and D = F^n - F^n_eq, the stages of Eq. (IMEX) for a tableau whose
// first stage is never advected reduce to (X_i = dt * L F^(i)):
//   dF1 = e1 D,  dF2 = e2 D,  F2 = F^n_eq + c2 D
//   R3 = F^n - k3 D - at32 X2                      F3 = R3 - a33 e3 D3
//   R4 = F^n - k4 D - at42 X2 - a43 e3 D3 - at43 X3,  F4 = R4 - a44 e4 D4
//   F^{n+1} = F^n - kf D - wt2 X2 - w3 e3 D3 - wt3 X3 - w4 e4 D4 - wt4 X4
// where D_i = R_i - F^(i)_eq and F^(i)_eq has the moments of R_i (Sec. III).
struct StageCoef {
  double k3, k4, kf;            // weights of D in R3, R4 and F^{n+1}
  double at32, at42, at43;      // explicit stage weights of X2, X3
  double wt2, wt3, wt4;         // explicit final weights
  double a33e3, a43e3, w3e3;    // weights of D3
  double a44e4, w4e4;           // weights of D4
  double c2;                    // F2 = F_eq + c2 (F - F_eq)
};

// One 1-D problem of a batch (fdlb_create_batch): its cells occupy
// [base, base + nx) of the concatenated population arrays.
struct BatchProblem {
  int64_t base;
  int nx;
  int pad_;
  double kchi, invDK;   // D+K-d and 1/(D+K) of this problem's gamma
  double dtdx;          // dt / dx
  double x0, x1;        // domain
  double split;         // membrane of the Riemann data in cell units (see
                        // split_in_cells): cell i is right of it iff i + 1/2 >= split
  double st[2][3];      // (rho, u, P) left and right
};

// Position of a membrane in cell units, s = (split - lo) n / (hi - lo), each
// operation rounded in binary64 in that order; cell i (centre lo + (i + 1/2)
// (hi - lo)/n) takes the right or upper state iff i + 1/2 >= s.  s is exact
// whenever the membrane sits on a cell face or centre of a grid whose length
// is a power of two times a small integer, in particular at the domain
// centre (s = n/2), so a cell centred there takes the right state as the
// Riemann set-up of Sec. V reads; comparing rounded centres instead lets the
// rounding of dx and of the centre move that cell to the left.
inline double split_in_cells(double split, double lo, double hi, int64_t n) {
  return ((split - lo) * (double)n) / (hi - lo);
}

// One tile of the batch work list: problem index and first cell.
struct WorkItem {
  int prob;
  int x0;
};

// Everything a stage kernel needs; passed by value as a __grid_constant__
// kernel parameter (about 14 KB).
struct DevParams {
  int d, nx, ny, bc;            // dimension, cells, boundary condition
  int Qp, Qc, P, nphi, nchi;    // lattice orders and population counts
  int64_t N;                    // cells = nx * ny
  double DK, kchi;              // D + K and D + K - d
  double dtdx, dtdy;            // dt/dx, dt/dy
  double pp[kMaxQ], pc[kMaxQ];  // phi and chi momenta (ascending)
  double wHp[kMaxQ * kMaxQ];    // [l*kMaxQ + k] = w_k He_l(p_k)/l!, phi axis
  double wHc[kMaxQ * kMaxQ];    // same for the chi axis
  // the same tables as binary32 pairs hi + lo (the mixed path's records)
  float wHph[kMaxQ * kMaxQ], wHpl[kMaxQ * kMaxQ], wHch[kMaxQ * kMaxQ], wHcl[kMaxQ * kMaxQ];
  double invDK;                 // 1 / (D + K)
  StageCoef sc;
  // per population: dt p_x/dx, dt p_y/dy, p_x, p_y, and p^2 (phi) or 0 (chi)
  double cx[kMaxPop], cy[kMaxPop], px[kMaxPop], py[kMaxPop], p2[kMaxPop];
  // binary32 splits p = hi + lo of p_x, p_y, p^2 (mixed precision moments)
  float pxh[kMaxPop], pxl[kMaxPop], pyh[kMaxPop], pyl[kMaxPop], p2h[kMaxPop], p2l[kMaxPop];
  int precision;  // FDLB_FP64 (double arrays) or FDLB_MIXED (float arrays)
  // Population arrays, element type double (FDLB_FP64) or float (FDLB_MIXED):
  void* F;      // state F^n (and F^{n+1} after the final stage)
  void* F2;     // stage-2 populations (advected by stage 3)
  void* F3;     // stage-3 populations (advected by stage 4); pass-1 scratch R3
  void* A4;     // stage-4 explicit part, then F4 (advected by the final stage)
  void* Af;     // running explicit part of F^{n+1}
  void* D;      // F^n - F^n_eq
  unsigned* status;  // bit 0: invalid moments seen
  // batches of 1-D problems (nprob > 0): N is the total cell count
  const BatchProblem* probs;
  const WorkItem* work;
  unsigned* pstatus;  // per problem: bit 0 invalid moments seen
  int nprob, nwork;
  int variant;  // 1-D tile shape of the batch kernels (0, 1, 2)
  int bgrid;    // persistent grid size of the batch kernels
  // FDLB_MIXED (fdlb_mixed.cu).  Each population of the state is an
  // unevaluated pair of binary32 values sh + sl (|sl| <= ulp(sh)/2), read
  // from (sh, sl) and written by the final stage to (nh, nl), the two buffers
  // swapping roles every step.  The stage arrays hold binary32 low parts
  // relative to the state's sh: R3 = sh + r3l, A4' = sh + a4l (then
  // R4 = sh + a4l), A_fin = sh + afl; dm holds D = R - F_eq of the last
  // stage; fa, fb, fc the low parts F2 - sh, F3 - sh, F4 - sh that stages 3,
  // 4 and final advect.  mhi[4][N] holds per cell the binary64 moment sums
  // (n, jx, jy, e) of sh.
  float *sh, *sl, *nh, *nl;
  float *r3l, *a4l, *afl;
  float *dm, *fa, *fb, *fc;
  double* mhi;
};

// 1-D tile shapes of the batch kernels, indexed by DevParams::variant:
// cells per tile and CTAs per SM of the persistent grid are the tuning knobs.
constexpr int kBatchVariants = 3;
int batch_tile_cells(int variant);

enum Stage { kPrep = 0, kStage3 = 1, kStage4 = 2, kFinal = 3 };

// Kernel launchers (fdlb_kernels.cu).  Each returns a cudaError_t value.
bool supported_lattice(int d, int Qp, int Qc);
int launch_stage(const DevParams& p, int stage, cudaStream_t s);
int launch_init_riemann(const DevParams& p, const double* states, int nq, double sx, double sy,
                        cudaStream_t s);
int launch_moments(const DevParams& p, double* n, double* ux, double* uy, double* T,
                   cudaStream_t s);
// J^T of the moment map at the binary64 state p.F (fdlb_moments_adjoint)
int launch_moments_adjoint(const DevParams& p, const double* nbar, const double* uxbar,
                           const double* uybar, const double* Tbar, double* Fbar, cudaStream_t s);
// batch kernels (d = 1, several problems in one launch)
int launch_batch_stage(const DevParams& p, int stage, cudaStream_t s);
int launch_batch_init(const DevParams& p, cudaStream_t s);
// binary32 stage kernels (fdlb_mixed.cu), single problems and batches;
// mixed_setup raises the kernels' shared-memory limit (call once before the
// first launch, outside stream capture)
int mixed_setup(const DevParams& p);
int launch_mixed_stage(const DevParams& p, int stage, cudaStream_t s);
int launch_mixed_batch_stage(const DevParams& p, int stage, cudaStream_t s);
// the binary32-pair state of FDLB_MIXED contexts <-> binary64 values
int launch_pair_to_double(const float* hi, const float* lo, double* out, int64_t n, cudaStream_t s);
int launch_double_to_pair(const double* in, float* hi, float* lo, int64_t n, cudaStream_t s);

}  // namespace fdlb
