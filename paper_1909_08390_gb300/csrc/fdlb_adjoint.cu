// fdlb_adjoint.cu -- discrete adjoint of the binary64 1-D IMEX step, hand
// written, with the MP limiter's selections frozen from the forward pass.
//
// Forward step (fused form, see fdlb_internal.h), per population array:
//   E0 = Feq(mom(F)), D = F - E0, F2 = E0 + c2 D, X2 = dt L(F2)
//   R3 = F - k3 D - at32 X2,  E3 = Feq(mom(R3)),  D3 = R3 - E3
//   F3 = R3 - a33e3 D3,  A4 = F - k4 D - at42 X2 - a43e3 D3,
//   Af = F - kf D - wt2 X2 - w3e3 D3,  X3 = dt L(F3)
//   R4 = A4 - at43 X3,  E4 = Feq(mom(R4)),  D4 = R4 - E4
//   F4 = R4 - a44e4 D4,  Af2 = Af - wt3 X3 - w4e4 D4,  X4 = dt L(F4)
//   F' = Af2 - wt4 X4.
// With the limiter's choices fixed, L is linear: each interface value is
// F_s plus one of the candidate offsets of Sec. IV (F^L - F_s, or a bound:
// 0, F_{s+1} - F_s, F^MD - F_s, F^UL - F_s, F^LC - F_s, with the four-way
// minmod choices inside F^MD and F^LC), each a fixed linear combination of
// the 9-cell window.  The adjoint kernels recompute those choices from the
// saved forward stage input with the forward's own integer-key comparisons
// and apply the transpose.  mom and Feq (Eq. Moments_discrete and
// Eq. gExpanded) are differentiated exactly: with a_l(u, T) the Hermite
// coefficients, da_l/du = l a_{l-1} and da_l/dT = l(l-1)/2 a_{l-2}.
// One adjoint kernel per advected stage (adj4, adj3, adj2) runs in reverse.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "fdlb.h"
#include "fdlb_ctx.h"
#include "fdlb_device.cuh"

namespace fdlb {
namespace {

constexpr int kTX = 16;   // cells per adjoint tile
constexpr int kNT = 128;  // threads per adjoint CTA
// Interfaces whose windows reach the tile's cells, per population: cell c
// lies in the windows of interfaces c-3 .. c+5 (p >= 0) or c-4 .. c+4
// (p < 0), so the tile needs [x0-3, x0+TX+4] or [x0-4, x0+TX+3].
constexpr int kNI = kTX + 8;
__device__ __forceinline__ int first_interface(int x0, int sgn) { return x0 - 4 + (sgn > 0 ? 1 : 0); }

// Scalar accumulators of the adjoint (binary64, device):
enum AdjScalar {
  kBarC2 = 0, kBarK3, kBarK4, kBarKf, kBarA33e3, kBarA43e3, kBarW3e3, kBarA44e4, kBarW4e4,
  kBarDK, kNumAdjScalars
};

struct AdjParams {
  const double* Fn;    // F^n of the step
  const double* F2s;   // stage-2 populations
  const double* F3s;   // stage-3 populations
  const double* F4s;   // stage-4 populations
  const double* Gbar;  // adjoint of F^{n+1}
  double* A4bar;       // adjoint of A4
  double* X3bar;       // adjoint of X3
  double* X2bar;       // adjoint of X2
  double* Fpart;       // direct part of the adjoint of F^n
  double* Dbar;        // adjoint of D
  double* Gnew;        // adjoint of F^n (output; may alias Gbar)
  double* scal;        // per block of the launch, kNumAdjScalars accumulators
};

// ---- frozen-limiter interface: value coefficients over the window ----------

// four-argument minmod choice (the value dm_bits returns): index 0..3 of the
// chosen argument, or -1 for zero
__device__ __forceinline__ int minmod4_choice(long long a, long long b, long long c, long long d) {
  const bool same = ((a ^ b) >= 0) && ((a ^ c) >= 0) && ((a ^ d) >= 0);
  const long long ma = a & kMag, mb = b & kMag, mc = c & kMag, md = d & kMag;
  const bool nz = (ma != 0) && (mb != 0) && (mc != 0) && (md != 0);
  int r = 0;
  long long mr = ma;
  if (mb < mr) { r = 1; mr = mb; }
  if (mc < mr) { r = 2; mr = mc; }
  if (md < mr) { r = 3; }
  return (same && nz) ? r : -1;
}

// coefficient vectors (over v[0..8] = F_{s-4..s+4}) of the curvatures
__device__ __forceinline__ void add_curv(double (&w)[9], int centre, double s) {
  // C_j = F_{j+1} - 2 F_j + F_{j-1}, centre j in window index
  w[centre - 1] += s;
  w[centre] -= 2.0 * s;
  w[centre + 1] += s;
}

// DM choice k over the pair (Ca at centre ca, Cb at centre cb) with the
// argument order (4Ca - Cb, 4Cb - Ca, Ca, Cb)
__device__ __forceinline__ void add_dm(double (&w)[9], int k, int ca, int cb, double s) {
  switch (k) {
    case 0: add_curv(w, ca, 4.0 * s); add_curv(w, cb, -s); break;
    case 1: add_curv(w, cb, 4.0 * s); add_curv(w, ca, -s); break;
    case 2: add_curv(w, ca, s); break;
    case 3: add_curv(w, cb, s); break;
    default: break;
  }
}

// Recompute the forward interface value of the window v (same operations and
// comparisons as mp9_face_fp64 inside the march) and return the coefficients
// w of the chosen linear expression: Fhat = sum_m w[m] v[m].
__device__ __forceinline__ void mp9_linearize(const double (&v)[9], double (&w)[9]) {
  using B = Mp9Coef;
  double d[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) d[k] = v[k + 1] - v[k];
  double a = B::b0 * d[0];
  a = fma(B::b1, d[1], a);
  a = fma(B::b2, d[2], a);
  a = fma(B::b3, d[3], a);
  a = fma(B::b4, d[4], a);
  a = fma(B::b5, d[5], a);
  a = fma(B::b6, d[6], a);
  a = fma(B::b7, d[7], a);
  const double cm1 = d[3] - d[2], c0 = d[4] - d[3], c1 = d[5] - d[4];
  // DM+ over (C_s, C_{s+1}); DM- as the march carries it: the DM+ of the
  // previous interface, over (C_{s-1}, C_s)
  const int kp = minmod4_choice(dbits(fma(4.0, c0, -c1)), dbits(fma(4.0, c1, -c0)), dbits(c0),
                                dbits(c1));
  const int km = minmod4_choice(dbits(fma(4.0, cm1, -c0)), dbits(fma(4.0, c0, -cm1)), dbits(cm1),
                                dbits(c0));
  // (selects, not indexed arrays, so that everything stays in registers)
  auto pick4 = [](int k, double x0, double x1, double x2, double x3) {
    return k == 0 ? x0 : k == 1 ? x1 : k == 2 ? x2 : k == 3 ? x3 : 0.0;
  };
  const double dmp = pick4(kp, fma(4.0, c0, -c1), fma(4.0, c1, -c0), c0, c1);
  const double dmm = pick4(km, fma(4.0, cm1, -c0), fma(4.0, c0, -cm1), cm1, c0);
  // candidate keys (twice their value), as in the forward
  enum { Z = 0, D0 = 1, MD = 2, UL = 3, LC = 4, A = 5 };
  const long long k_d0 = key_times_pow2<1>(dbits(d[4]));
  const long long k_md = okey(dbits(d[4] - dmp));
  const long long k_ul = key_times_pow2<3>(dbits(d[3]));
  const long long k_lc = okey(dbits(fma(8.0 / 3.0, dmm, d[3])));
  const long long ka = key_times_pow2<1>(dbits(a));
  auto key = [&](int i) {
    return i == D0 ? k_d0 : i == MD ? k_md : i == UL ? k_ul : i == LC ? k_lc : i == A ? ka : 0LL;
  };
  // lo = kmax(kmin(0, kmin(k_d0, k_md)), kmin(0, kmin(k_ul, k_lc))), with the
  // forward's tie rules: kmin(a, b) = a < b ? a : b, kmax(a, b) = a < b ? b : a
  auto kmin_i = [&](int i, int j) { return key(i) < key(j) ? i : j; };
  auto kmax_i = [&](int i, int j) { return key(i) < key(j) ? j : i; };
  const int lo = kmax_i(kmin_i(Z, kmin_i(D0, MD)), kmin_i(Z, kmin_i(UL, LC)));
  const int hi = kmin_i(kmax_i(Z, kmax_i(D0, MD)), kmax_i(Z, kmax_i(UL, LC)));
  // r = kmin(kmax(ka, lo), hi)
  int sel = (ka < key(lo)) ? lo : A;
  if (!(key(sel) < key(hi))) sel = hi;
#pragma unroll
  for (int m = 0; m < 9; ++m) w[m] = 0.0;
  w[4] = 1.0;  // F_s
  switch (sel) {
    case A: {
      const double b[8] = {B::b0, B::b1, B::b2, B::b3, B::b4, B::b5, B::b6, B::b7};
#pragma unroll
      for (int m = 0; m < 9; ++m) w[m] += (m > 0 ? b[m - 1] : 0.0) - (m < 8 ? b[m] : 0.0);
      break;
    }
    case D0: w[5] += 1.0; w[4] -= 1.0; break;
    case MD:  // (d_0 - DM+)/2
      w[5] += 0.5; w[4] -= 0.5;
      add_dm(w, kp, 4, 5, -0.5);
      break;
    case UL: w[4] += 4.0; w[3] -= 4.0; break;
    case LC:  // d_-1/2 + (4/3) DM-
      w[4] += 0.5; w[3] -= 0.5;
      add_dm(w, km, 3, 4, 4.0 / 3.0);
      break;
    default: break;  // Z: F_s
  }
}

// ---- equilibrium Jacobian ------------------------------------------------

// One axis of the equilibrium factors and their u- and T-derivatives
// (Eq. gExpanded): g_k = sum_l c_lk a_l, dg_k/du = sum_l c_lk l a_{l-1},
// dg_k/dT = sum_l c_lk l(l-1)/2 a_{l-2}, with c_lk = w_k He_l(p_k)/l!.  The
// nodes are antisymmetric, so each sum splits into even and odd l and gives
// the mirror node (Q-1-k) from the same partial sums.
template <int Q>
__device__ __forceinline__ void axis_g_derivs(const double* wH, double u, double T, double (&g)[Q],
                                              double (&gu)[Q], double (&gT)[Q]) {
  double a[Q];
  a[0] = 1.0;
  if (Q > 1) a[1] = u;
  const double tm1 = T - 1.0;
#pragma unroll
  for (int l = 2; l < Q; ++l) a[l] = fma(u, a[l - 1], ((double)(l - 1) * tm1) * a[l - 2]);
#pragma unroll
  for (int k = 0; k < (Q + 1) / 2; ++k) {
    double ge = 0.0, go = 0.0, ue = 0.0, uo = 0.0, te = 0.0, to = 0.0;
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      const double c = wH[l * kMaxQ + k];
      // even/odd: by the parity of l, which fixes the sign at the mirror node
      if (l & 1) {
        go = fma(c, a[l], go);
        uo = fma(c * (double)l, a[l - 1], uo);
        if (l >= 2) to = fma(c * (0.5 * l * (l - 1)), a[l - 2], to);
      } else {
        ge = fma(c, a[l], ge);
        if (l >= 1) ue = fma(c * (double)l, a[l - 1], ue);
        if (l >= 2) te = fma(c * (0.5 * l * (l - 1)), a[l - 2], te);
      }
    }
    // parity in p_k: c_{l,Q-1-k} = (-1)^l c_lk
    g[k] = ge + go;
    gu[k] = ue + uo;
    gT[k] = te + to;
    if (Q - 1 - k != k) {
      g[Q - 1 - k] = ge - go;
      gu[Q - 1 - k] = ue - uo;
      gT[Q - 1 - k] = te - to;
    }
  }
}

// Adjoints of a cell's moment sums n, j, e (so that R's populations receive
// rn + rj p + re p^2 (phi) or re (chi)) and of D + K at fixed moment sums.
struct EqAdj {
  double rn, rj, re;
  double dk;
};

// ---- the three adjoint stage kernels -------------------------------------

// Shared memory: per population, the frozen-limiter weights of the tile's
// interfaces over their 9 window cells and the adjoint each interface
// receives; the gathered adjoint of the advected array; and the Hermite
// coefficient tables of the equilibrium derivatives, c_lk l and
// c_lk l(l-1)/2 (c_lk = w_k He_l(p_k)/l!), formed once per CTA.
template <int QP, int QC>
struct AdjSmem {
  static constexpr int P = QP + QC;
  double wts[P][kNI][9];
  double ifb[P][kNI];
  double fbar[P][kTX];
  double cup[QP * QP], cTp[QP * QP], cuc[QC * QC], cTc[QC * QC];
};

template <int QP, int QC>
__device__ __forceinline__ void fill_deriv_tables(const DevParams& p, AdjSmem<QP, QC>& sm) {
  for (int t = threadIdx.x; t < QP * QP + QC * QC; t += kNT) {
    const bool phi = t < QP * QP;
    const int Q = phi ? QP : QC;
    const int lk = phi ? t : t - QP * QP;
    const int l = lk / Q, k = lk % Q;
    const double c = (phi ? p.wHp : p.wHc)[l * kMaxQ + k];
    (phi ? sm.cup : sm.cuc)[lk] = c * (double)l;
    (phi ? sm.cTp : sm.cTc)[lk] = c * (0.5 * l * (l - 1));
  }
}

__device__ __forceinline__ int clampi(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

// Window cell of slot m for interface i (between cells i-1 and i) and sign.
__device__ __forceinline__ int slot_cell(int i, int m, int sgn) {
  return sgn > 0 ? (i - 1) + (m - 4) : i - (m - 4);
}

// dt L^T: the adjoint of X = dt L(Fin) for the tile's cells, every population,
// into sm.fbar (each interface's adjoint times its window weights, summed).
// Xbar(pop, cell) gives the adjoint of X at any cell.
template <int QP, int QC, typename XbarFn>
__device__ __forceinline__ void advect_adjoint(const DevParams& p, const double* Fin, int x0,
                                               AdjSmem<QP, QC>& sm, XbarFn Xbar) {
  constexpr int P = QP + QC;
  const int nx = p.nx;
  const int64_t N = p.N;
  const int tid = threadIdx.x;
  for (int t = tid; t < P * kNI; t += kNT) {
    const int pop = t / kNI;
    const int ii = t % kNI;
    const double px = p.px[pop];
    const int sgn = px >= 0.0 ? 1 : -1;
    const int i = first_interface(x0, sgn) + ii;  // interface index
    double* c = sm.wts[pop][ii];
    if (i < 0 || i > nx) {
#pragma unroll
      for (int m = 0; m < 9; ++m) c[m] = 0.0;
      sm.ifb[pop][ii] = 0.0;
      continue;
    }
    double v[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) v[m] = Fin[pop * N + clampi(slot_cell(i, m, sgn), nx)];
    double w[9];
    mp9_linearize(v, w);
    // X_c = (dt p / dx) (Fhat_{c+1} - Fhat_c): Fhat_i enters X_{i-1} with +, X_i with -
    const double cp = p.dtdx * px;
    const double xl = (i - 1 >= 0) ? Xbar(pop, i - 1) : 0.0;
    const double xr = (i <= nx - 1) ? Xbar(pop, i) : 0.0;
    sm.ifb[pop][ii] = cp * (xl - xr);
#pragma unroll
    for (int m = 0; m < 9; ++m) c[m] = w[m];
  }
  __syncthreads();
  // gather: cell c sits at slot m = c - i + 5 of interface i (p >= 0, i in
  // [c-3, c+5]) or m = i + 4 - c (p < 0, i in [c-4, c+4]); the clamped ghost
  // slots of the first and last interfaces add to cells 0 and nx-1
  for (int t = tid; t < P * kTX; t += kNT) {
    const int pop = t / kTX;
    const int lc = t % kTX;
    const int cell = x0 + lc;
    double acc = 0.0;
    if (cell < nx) {
      const int sgn = p.px[pop] >= 0.0 ? 1 : -1;
      const int ifirst = sgn > 0 ? cell - 3 : cell - 4;
      const int ibase = first_interface(x0, sgn);
#pragma unroll
      for (int t9 = 0; t9 < 9; ++t9) {
        const int i = ifirst + t9;
        const int m = sgn > 0 ? cell - i + 5 : i + 4 - cell;
        if (i >= 0 && i <= nx) {
          const int ii = i - ibase;
          acc = fma(sm.ifb[pop][ii], sm.wts[pop][ii][m], acc);
        }
      }
      if (cell == 0 || cell == nx - 1) {
        // slots whose window cell lies outside [0, nx) and is clamped to `cell`
        for (int i = (cell == 0 ? 0 : nx - 4); i <= (cell == 0 ? 4 : nx); ++i) {
          if (i < 0 || i > nx) continue;
#pragma unroll
          for (int m = 0; m < 9; ++m) {
            const int sc = slot_cell(i, m, sgn);
            if ((cell == 0 && sc < 0) || (cell == nx - 1 && sc > nx - 1))
              acc = fma(sm.ifb[pop][i - ibase], sm.wts[pop][i - ibase][m], acc);
          }
        }
      }
    }
    sm.fbar[pop][lc] = acc;
  }
  __syncthreads();
}

// Adds the block's sums of v[i] to row[id[i]], this block's own row of
// accumulators: a shuffle tree in each warp, then the warps' sums in warp
// order.  No atomics, so the sums are the same on every run.  Every thread
// of the block calls it (it holds a barrier); blockDim.x is a multiple of 32.
template <int N>
__device__ __forceinline__ void block_accumulate(double* __restrict__ row, const int (&id)[N],
                                                 double (&v)[N]) {
  __shared__ double ws[N][32];
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    if ((threadIdx.x & 31) == 0) ws[i][warp] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < N) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += ws[threadIdx.x][w];
    row[id[threadIdx.x]] += t;
  }
}

// ---- per-cell phases: 8 threads per cell ---------------------------------
// The 128 threads of a tile take its 16 cells 8 at a time: sub-thread s of a
// cell owns populations s and s + 8, evaluates the equilibrium factor and its
// derivatives of its own nodes, and the cell's sums (moments, equilibrium
// adjoint) are reduced over the 8 lanes with shuffles.
constexpr int kSub = 8;
static_assert(kTX * kSub == kNT, "8 threads per cell");

// sum over the 8 lanes of a cell (aligned groups of 8 within the warp)
__device__ __forceinline__ double cell_sum(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

// One node's equilibrium factor and its u- and T-derivatives (Eq. gExpanded),
// with the derivative coefficients c_lk l and c_lk l(l-1)/2 from the tables.
template <int Q>
__device__ __forceinline__ void node_derivs(const double* wH, const double* cu, const double* cT,
                                            int k, double u, double T, double& g, double& gu,
                                            double& gT) {
  double a[Q];
  a[0] = 1.0;
  if (Q > 1) a[1] = u;
  const double tm1 = T - 1.0;
#pragma unroll
  for (int l = 2; l < Q; ++l) a[l] = fma(u, a[l - 1], ((double)(l - 1) * tm1) * a[l - 2]);
  g = 0.0;
  gu = 0.0;
  gT = 0.0;
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    g = fma(wH[l * kMaxQ + k], a[l], g);
    if (l >= 1) gu = fma(cu[l * Q + k], a[l - 1], gu);
    if (l >= 2) gT = fma(cT[l * Q + k], a[l - 2], gT);
  }
}

// A population's equilibrium and the factors its adjoint needs.
struct PopEq {
  double fe;          // the equilibrium population
  double dn, du, dT;  // its derivatives with respect to n, u, T
  double dk;          // its derivative with respect to D + K at fixed n, u, T
};

__device__ __forceinline__ PopEq phi_eq(double n, double g, double gu, double gT) {
  return PopEq{n * g, g, n * gu, n * gT, 0.0};
}
__device__ __forceinline__ PopEq chi_eq(double kc, double n, double T, double g, double gu,
                                        double gT) {
  // chi^eq = (D+K-d) T n h
  return PopEq{kc * T * n * g, kc * T * g, kc * T * n * gu, kc * n * (g + T * gT), T * n * g};
}

// The equilibria of the sub-thread's populations sub and sub + kSub.  On the
// (8, 8) lattice they are the phi and chi populations of one node, whose
// factors are evaluated once.
template <int QP, int QC>
__device__ __forceinline__ void pop_eqs(const DevParams& p, const AdjSmem<QP, QC>& sm, int sub,
                                        double n, double u, double T, PopEq (&q)[2]) {
  constexpr int P = QP + QC;
  double g, gu, gT;
  if constexpr (QP == QC && QP == kSub) {
    node_derivs<QP>(p.wHp, sm.cup, sm.cTp, sub, u, T, g, gu, gT);
    q[0] = phi_eq(n, g, gu, gT);
    q[1] = chi_eq(p.kchi, n, T, g, gu, gT);
  } else {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int pop = sub + kSub * r;
      if (pop >= P) break;
      if (pop < QP) {
        node_derivs<QP>(p.wHp, sm.cup, sm.cTp, pop, u, T, g, gu, gT);
        q[r] = phi_eq(n, g, gu, gT);
      } else {
        node_derivs<QC>(p.wHc, sm.cuc, sm.cTc, pop - QP, u, T, g, gu, gT);
        q[r] = chi_eq(p.kchi, n, T, g, gu, gT);
      }
    }
  }
}

// The cell's (n, j, e) from the sub-thread's populations v[0..1].
template <int QP, int QC>
__device__ __forceinline__ void cell_moments(const DevParams& p, int sub, const double (&v)[2],
                                             double& n, double& j, double& e) {
  n = 0.0;
  j = 0.0;
  e = 0.0;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int pop = sub + kSub * r;
    if (pop >= QP + QC) break;
    if (pop < QP) {
      n += v[r];
      j = fma(p.px[pop], v[r], j);
      e = fma(p.p2[pop], v[r], e);
    } else {
      e += v[r];
    }
  }
  n = cell_sum(n);
  j = cell_sum(j);
  e = cell_sum(e);
}

// Adjoint of (n, j, e) -> (n, u, T), u = j/n, T = (e - j^2/n)/((D+K) n):
// from the cell's reduced adjoints of n, u, T and of D+K at fixed (n, u, T)
// to those of the moment sums and of D+K at fixed moment sums.
__device__ __forceinline__ EqAdj moments_adjoint(const DevParams& p, double n, double u, double T,
                                                 double e, double nb, double ub, double Tb,
                                                 double kb) {
  const double inv_n = 1.0 / n, DK = p.DK;
  EqAdj r;
  r.rn = nb - ub * u * inv_n + Tb * (2.0 * n * u * u - e) * inv_n * inv_n / DK;
  r.rj = ub * inv_n - Tb * 2.0 * u * inv_n / DK;
  r.re = Tb * inv_n / DK;
  r.dk = -Tb * T / DK + kb;  // T = (...)/DK and kchi = DK - d
  return r;
}

// Stage 4 + final: from Gbar = adjoint of F^{n+1}.
template <int QP, int QC>
__global__ void __launch_bounds__(kNT) adj4_kernel(const __grid_constant__ DevParams p,
                                                   const __grid_constant__ AdjParams a) {
  constexpr int P = QP + QC;
  __shared__ AdjSmem<QP, QC> sm;
  const StageCoef& sc = p.sc;
  const int x0 = blockIdx.x * kTX;
  fill_deriv_tables<QP, QC>(p, sm);  // read after advect_adjoint's barriers
  const int64_t N = p.N;
  // X4bar = -wt4 Gbar
  advect_adjoint<QP, QC>(p, a.F4s, x0, sm,
                         [&](int pop, int c) { return -sc.wt4 * a.Gbar[pop * N + c]; });
  const int lc = threadIdx.x / kSub, sub = threadIdx.x % kSub;
  const int cell = x0 + lc;
  const bool live = cell < p.nx;
  double s_a44 = 0.0, s_w4 = 0.0, s_dk = 0.0;
  double F4[2] = {0.0, 0.0};
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int pop = sub + kSub * r;
    if (live && pop < P) F4[r] = a.F4s[pop * N + cell];
  }
  double n, j, e;
  cell_moments<QP, QC>(p, sub, F4, n, j, e);  // moments of F4 = moments of R4
  if (!live) n = 1.0;                         // a harmless dummy cell
  const double inv_n = 1.0 / n, u = j * inv_n, T = (e - n * u * u) * inv_n * p.invDK;
  const double inv = 1.0 / (1.0 - sc.a44e4);
  double R4b[2] = {0.0, 0.0}, G[2] = {0.0, 0.0};
  PopEq q[2];
  pop_eqs<QP, QC>(p, sm, sub, n, u, T, q);
  double nb = 0.0, ub = 0.0, Tb = 0.0, kb = 0.0;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int pop = sub + kSub * r;
    if (pop >= P || !live) break;
    G[r] = a.Gbar[pop * N + cell];
    const double f4b = sm.fbar[pop][lc];
    const double D4 = (F4[r] - q[r].fe) * inv;  // R4 - E4
    R4b[r] = (1.0 - sc.a44e4) * f4b - sc.w4e4 * G[r];
    const double eb = sc.a44e4 * f4b + sc.w4e4 * G[r];
    s_a44 -= f4b * D4;
    s_w4 -= G[r] * D4;
    nb = fma(eb, q[r].dn, nb);
    ub = fma(eb, q[r].du, ub);
    Tb = fma(eb, q[r].dT, Tb);
    kb = fma(eb, q[r].dk, kb);
  }
  const EqAdj ea = moments_adjoint(p, n, u, T, e, cell_sum(nb), cell_sum(ub), cell_sum(Tb),
                                   cell_sum(kb));
  if (sub == 0 && live) s_dk = ea.dk;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int pop = sub + kSub * r;
    if (pop >= P || !live) break;
    const double rb = R4b[r] + (pop < QP ? fma(p.p2[pop], ea.re, fma(p.px[pop], ea.rj, ea.rn)) : ea.re);
    a.A4bar[pop * N + cell] = rb;
    a.X3bar[pop * N + cell] = -sc.wt3 * G[r] - sc.at43 * rb;
  }
  {
    const int id[3] = {kBarA44e4, kBarW4e4, kBarDK};
    double v[3] = {s_a44, s_w4, s_dk};
    block_accumulate<3>(a.scal + (int64_t)blockIdx.x * kNumAdjScalars, id, v);
  }
}

// Stage 3.
template <int QP, int QC>
__global__ void __launch_bounds__(kNT) adj3_kernel(const __grid_constant__ DevParams p,
                                                   const __grid_constant__ AdjParams a) {
  constexpr int P = QP + QC;
  __shared__ AdjSmem<QP, QC> sm;
  const StageCoef& sc = p.sc;
  const int x0 = blockIdx.x * kTX;
  fill_deriv_tables<QP, QC>(p, sm);  // read after advect_adjoint's barriers
  const int64_t N = p.N;
  advect_adjoint<QP, QC>(p, a.F3s, x0, sm, [&](int pop, int c) { return a.X3bar[pop * N + c]; });
  const int lc = threadIdx.x / kSub, sub = threadIdx.x % kSub;
  const int cell = x0 + lc;
  const bool live = cell < p.nx;
  double s[7] = {0, 0, 0, 0, 0, 0, 0};  // a33e3 a43e3 w3e3 k3 k4 kf dk
  // relaxation of stage 3: F3 = R3 - a33e3 D3, D3 = R3 - F_eq(m(R3))
  double F3[2] = {0.0, 0.0}, Fn[2] = {0.0, 0.0};
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int pop = sub + kSub * r;
    if (live && pop < P) {
      F3[r] = a.F3s[pop * N + cell];
      Fn[r] = a.Fn[pop * N + cell];
    }
  }
  double n, j, e, n0, j0, e0;
  cell_moments<QP, QC>(p, sub, F3, n, j, e);
  cell_moments<QP, QC>(p, sub, Fn, n0, j0, e0);
  if (!live) n = n0 = 1.0;
  const double inv_n = 1.0 / n, u = j * inv_n, T = (e - n * u * u) * inv_n * p.invDK;
  const double inv_n0 = 1.0 / n0, u0 = j0 * inv_n0, T0 = (e0 - n0 * u0 * u0) * inv_n0 * p.invDK;
  const double inv = 1.0 / (1.0 - sc.a33e3);
  double R3b[2] = {0.0, 0.0}, A4b[2] = {0.0, 0.0}, G[2] = {0.0, 0.0};
  double nb = 0.0, ub = 0.0, Tb = 0.0, kb = 0.0;
  PopEq qs[2];
  pop_eqs<QP, QC>(p, sm, sub, n, u, T, qs);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int pop = sub + kSub * r;
    if (pop >= P || !live) break;
    const PopEq& q = qs[r];
    A4b[r] = a.A4bar[pop * N + cell];
    G[r] = a.Gbar[pop * N + cell];
    const double f3b = sm.fbar[pop][lc];
    const double D3 = (F3[r] - q.fe) * inv;
    R3b[r] = (1.0 - sc.a33e3) * f3b - sc.a43e3 * A4b[r] - sc.w3e3 * G[r];
    const double eb = sc.a33e3 * f3b + sc.a43e3 * A4b[r] + sc.w3e3 * G[r];
    s[0] -= f3b * D3;
    s[1] -= A4b[r] * D3;
    s[2] -= G[r] * D3;
    nb = fma(eb, q.dn, nb);
    ub = fma(eb, q.du, ub);
    Tb = fma(eb, q.dT, Tb);
    kb = fma(eb, q.dk, kb);
  }
  const EqAdj ea = moments_adjoint(p, n, u, T, e, cell_sum(nb), cell_sum(ub), cell_sum(Tb),
                                   cell_sum(kb));
  if (sub == 0 && live) s[6] = ea.dk;
  // explicit part R3 = F - k3 D - at32 X2, A4 and A_fin: adjoints of F, D, X2
  PopEq q0[2];
  pop_eqs<QP, QC>(p, sm, sub, n0, u0, T0, q0);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int pop = sub + kSub * r;
    if (pop >= P || !live) break;
    const double e0p = q0[r].fe;
    const double rb = R3b[r] + (pop < QP ? fma(p.p2[pop], ea.re, fma(p.px[pop], ea.rj, ea.rn)) : ea.re);
    const double D = Fn[r] - e0p;
    s[3] -= rb * D;
    s[4] -= A4b[r] * D;
    s[5] -= G[r] * D;
    a.Fpart[pop * N + cell] = rb + A4b[r] + G[r];
    a.Dbar[pop * N + cell] = -sc.k3 * rb - sc.k4 * A4b[r] - sc.kf * G[r];
    a.X2bar[pop * N + cell] = -sc.at32 * rb - sc.at42 * A4b[r] - sc.wt2 * G[r];
  }
  {
    const int id[7] = {kBarA33e3, kBarA43e3, kBarW3e3, kBarK3, kBarK4, kBarKf, kBarDK};
    block_accumulate<7>(a.scal + (int64_t)blockIdx.x * kNumAdjScalars, id, s);
  }
}

// Stage 2 (and the stage-1/2 closed forms): adjoint of F^n.
template <int QP, int QC>
__global__ void __launch_bounds__(kNT) adj2_kernel(const __grid_constant__ DevParams p,
                                                   const __grid_constant__ AdjParams a) {
  constexpr int P = QP + QC;
  __shared__ AdjSmem<QP, QC> sm;
  const StageCoef& sc = p.sc;
  const int x0 = blockIdx.x * kTX;
  fill_deriv_tables<QP, QC>(p, sm);  // read after advect_adjoint's barriers
  const int64_t N = p.N;
  advect_adjoint<QP, QC>(p, a.F2s, x0, sm, [&](int pop, int c) { return a.X2bar[pop * N + c]; });
  const int lc = threadIdx.x / kSub, sub = threadIdx.x % kSub;
  const int cell = x0 + lc;
  const bool live = cell < p.nx;
  double s_c2 = 0.0, s_dk = 0.0;
  double Fn[2] = {0.0, 0.0};
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int pop = sub + kSub * r;
    if (live && pop < P) Fn[r] = a.Fn[pop * N + cell];
  }
  double n0, j0, e0;
  cell_moments<QP, QC>(p, sub, Fn, n0, j0, e0);
  if (!live) n0 = 1.0;
  const double inv_n0 = 1.0 / n0, u0 = j0 * inv_n0, T0 = (e0 - n0 * u0 * u0) * inv_n0 * p.invDK;
  double Dt[2] = {0.0, 0.0};
  double nb = 0.0, ub = 0.0, Tb = 0.0, kb = 0.0;
  PopEq qs[2];
  pop_eqs<QP, QC>(p, sm, sub, n0, u0, T0, qs);
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int pop = sub + kSub * r;
    if (pop >= P || !live) break;
    const PopEq& q = qs[r];
    const double f2b = sm.fbar[pop][lc];
    Dt[r] = a.Dbar[pop * N + cell] + sc.c2 * f2b;  // total adjoint of D
    const double eb = f2b - Dt[r];                  // F2 = E0 + c2 D, D = F - E0
    s_c2 += f2b * (Fn[r] - q.fe);
    nb = fma(eb, q.dn, nb);
    ub = fma(eb, q.du, ub);
    Tb = fma(eb, q.dT, Tb);
    kb = fma(eb, q.dk, kb);
  }
  const EqAdj ea = moments_adjoint(p, n0, u0, T0, e0, cell_sum(nb), cell_sum(ub), cell_sum(Tb),
                                   cell_sum(kb));
  if (sub == 0 && live) s_dk = ea.dk;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int pop = sub + kSub * r;
    if (pop >= P || !live) break;
    const double rb = pop < QP ? fma(p.p2[pop], ea.re, fma(p.px[pop], ea.rj, ea.rn)) : ea.re;
    a.Gnew[pop * N + cell] = a.Fpart[pop * N + cell] + Dt[r] + rb;
  }
  {
    const int id[2] = {kBarC2, kBarDK};
    double v[2] = {s_c2, s_dk};
    block_accumulate<2>(a.scal + (int64_t)blockIdx.x * kNumAdjScalars, id, v);
  }
}

// ---- initial fields and their adjoint ---------------------------------------

template <int QP, int QC>
__global__ void init_fields_kernel(const __grid_constant__ DevParams p, const double* __restrict__ n,
                                   const double* __restrict__ u, const double* __restrict__ T) {
  constexpr int P = QP + QC;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  const double nn = n[c], uu = u[c], TT = T[c];
  // moment sums of the equilibrium of (n, u, T): j = n u, e = n u^2 + (D+K) n T
  double Feq[P];
  double g[QP], gu[QP], gT[QP];
  axis_g_derivs<QP>(p.wHp, uu, TT, g, gu, gT);
  double h[QC], hu[QC], hT[QC];
  axis_g_derivs<QC>(p.wHc, uu, TT, h, hu, hT);
#pragma unroll
  for (int k = 0; k < QP; ++k) Feq[k] = nn * g[k];
#pragma unroll
  for (int q = 0; q < QC; ++q) Feq[QP + q] = p.kchi * TT * nn * h[q];
  double* F = (double*)p.F;
#pragma unroll
  for (int k = 0; k < P; ++k) F[k * p.N + c] = Feq[k];
}

template <int QP, int QC>
__global__ void init_fields_adjoint_kernel(const __grid_constant__ DevParams p,
                                           const double* __restrict__ Fbar,
                                           const double* __restrict__ n,
                                           const double* __restrict__ u,
                                           const double* __restrict__ T, double* __restrict__ nb,
                                           double* __restrict__ ub, double* __restrict__ Tb,
                                           double* __restrict__ dkbar) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s_dk = 0.0;
  if (c < p.N) {
    const double nn = n[c], uu = u[c], TT = T[c];
    double g[QP], gu[QP], gT[QP];
    axis_g_derivs<QP>(p.wHp, uu, TT, g, gu, gT);
    double h[QC], hu[QC], hT[QC];
    axis_g_derivs<QC>(p.wHc, uu, TT, h, hu, hT);
    double sn = 0.0, su = 0.0, sT = 0.0;
#pragma unroll
    for (int k = 0; k < QP; ++k) {
      const double fb = Fbar[k * p.N + c];
      sn = fma(fb, g[k], sn);
      su = fma(fb, nn * gu[k], su);
      sT = fma(fb, nn * gT[k], sT);
    }
#pragma unroll
    for (int q = 0; q < QC; ++q) {
      const double fb = Fbar[(QP + q) * p.N + c];
      sn = fma(fb, p.kchi * TT * h[q], sn);
      su = fma(fb, p.kchi * TT * nn * hu[q], su);
      sT = fma(fb, p.kchi * nn * (h[q] + TT * hT[q]), sT);
      s_dk = fma(fb, TT * nn * h[q], s_dk);  // chi^eq = (D+K-d) T n h
    }
    nb[c] = sn;
    ub[c] = su;
    Tb[c] = sT;
  }
  const int id[1] = {0};
  double v[1] = {s_dk};
  block_accumulate<1>(dkbar + blockIdx.x, id, v);
}

}  // namespace
}  // namespace fdlb

// ---- host side ------------------------------------------------------------------

namespace {

using fdlb::DevParams;

bool adjoint_lattice(const fdlb_ctx* c) {
  return !c->batch && !c->custom_tableau && c->dp.d == 1 && c->precision == FDLB_FP64 &&
         ((c->dp.Qp == 8 && c->dp.Qc == 8) || (c->dp.Qp == 5 && c->dp.Qc == 3) ||
          (c->dp.Qp == 3 && c->dp.Qc == 3)) &&
         c->dp.bc == FDLB_BC_OUTLET;
}

template <int QP, int QC>
int launch_adj(int which, const DevParams& p, const fdlb::AdjParams& a, cudaStream_t s) {
  const int nb = (p.nx + fdlb::kTX - 1) / fdlb::kTX;
  if (which == 4) fdlb::adj4_kernel<QP, QC><<<nb, fdlb::kNT, 0, s>>>(p, a);
  else if (which == 3) fdlb::adj3_kernel<QP, QC><<<nb, fdlb::kNT, 0, s>>>(p, a);
  else fdlb::adj2_kernel<QP, QC><<<nb, fdlb::kNT, 0, s>>>(p, a);
  return (int)cudaGetLastError();
}

int launch_adj_any(int which, const DevParams& p, const fdlb::AdjParams& a, cudaStream_t s) {
  if (p.Qp == 8) return launch_adj<8, 8>(which, p, a, s);
  if (p.Qp == 5) return launch_adj<5, 3>(which, p, a, s);
  return launch_adj<3, 3>(which, p, a, s);
}

// Derivatives of the fused stage coefficients with respect to lam = dt/tau,
// for the paper's tableau (the only one the adjoint supports).
void stage_coef_dlam(double lam, double* dc) {
  const double al = 0.24169426078821, be = 0.06042356519705, et = 0.12915286960590;
  const double A[4][4] = {{al, 0, 0, 0}, {-al, al, 0, 0}, {0, 1 - al, al, 0},
                          {be, et, 0.5 - be - et - al, al}};
  const double w[4] = {0.0, 1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
  double e[4], de[4];
  for (int i = 0; i < 4; ++i) {
    const double den = 1.0 + A[i][i] * lam;
    e[i] = lam / den;
    de[i] = 1.0 / (den * den);
  }
  const double d1 = e[0], dd1 = de[0];
  const double d2 = e[1] * (1.0 - A[1][0] * d1);
  const double dd2 = de[1] * (1.0 - A[1][0] * d1) - e[1] * A[1][0] * dd1;
  (void)d2;
  dc[fdlb::kBarC2] = -A[1][0] * dd1 - A[1][1] * dd2;
  dc[fdlb::kBarK3] = A[2][0] * dd1 + A[2][1] * dd2;
  dc[fdlb::kBarK4] = A[3][0] * dd1 + A[3][1] * dd2;
  dc[fdlb::kBarKf] = w[0] * dd1 + w[1] * dd2;
  dc[fdlb::kBarA33e3] = A[2][2] * de[2];
  dc[fdlb::kBarA43e3] = A[3][2] * de[2];
  dc[fdlb::kBarW3e3] = w[2] * de[2];
  dc[fdlb::kBarA44e4] = A[3][3] * de[3];
  dc[fdlb::kBarW4e4] = w[3] * de[3];
}

}  // namespace

extern "C" {

int fdlb_init_fields(fdlb_ctx* c, const double* n, const double* u, const double* T) {
  if (!c || !n || !u || !T) return fdlb::ctx_error(c, FDLB_EINVAL, "NULL argument");
  if (!adjoint_lattice(c))
    return fdlb::ctx_error(c, FDLB_EINVAL, "fdlb_init_fields: 1-D binary64 outlet contexts");
  const int nt = 128;
  const int64_t nb = (c->dp.N + nt - 1) / nt;
  if (c->dp.Qp == 8) fdlb::init_fields_kernel<8, 8><<<(unsigned)nb, nt, 0, c->stream>>>(c->dp, n, u, T);
  else if (c->dp.Qp == 5) fdlb::init_fields_kernel<5, 3><<<(unsigned)nb, nt, 0, c->stream>>>(c->dp, n, u, T);
  else fdlb::init_fields_kernel<3, 3><<<(unsigned)nb, nt, 0, c->stream>>>(c->dp, n, u, T);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fdlb::ctx_error(c, FDLB_ECUDA, cudaGetErrorString(e));
  c->prepared = false;
  return fdlb::ctx_prepare(c);
}

int fdlb_init_fields_adjoint(fdlb_ctx* c, const double* Fbar, const double* n, const double* u,
                             const double* T, double* nbar, double* ubar, double* Tbar,
                             double* dgamma) {
  if (!c || !Fbar || !n || !u || !T || !nbar || !ubar || !Tbar || !dgamma)
    return fdlb::ctx_error(c, FDLB_EINVAL, "NULL argument");
  if (!adjoint_lattice(c))
    return fdlb::ctx_error(c, FDLB_EINVAL, "fdlb_init_fields_adjoint: 1-D binary64 outlet contexts");
  // one D+K adjoint accumulator per block, summed here in block order
  const int nt = 128;
  const int64_t nb = (c->dp.N + nt - 1) / nt;
  std::vector<double> hd((size_t)nb, 0.0);
  double* dk = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&dk, (size_t)nb * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(dk, 0, (size_t)nb * sizeof(double), c->stream);
  if (e != cudaSuccess) return fdlb::ctx_error(c, FDLB_ECUDA, cudaGetErrorString(e));
  if (c->dp.Qp == 8)
    fdlb::init_fields_adjoint_kernel<8, 8><<<(unsigned)nb, nt, 0, c->stream>>>(c->dp, Fbar, n, u, T, nbar, ubar, Tbar, dk);
  else if (c->dp.Qp == 5)
    fdlb::init_fields_adjoint_kernel<5, 3><<<(unsigned)nb, nt, 0, c->stream>>>(c->dp, Fbar, n, u, T, nbar, ubar, Tbar, dk);
  else
    fdlb::init_fields_adjoint_kernel<3, 3><<<(unsigned)nb, nt, 0, c->stream>>>(c->dp, Fbar, n, u, T, nbar, ubar, Tbar, dk);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hd.data(), dk, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(dk, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fdlb::ctx_error(c, FDLB_ECUDA, cudaGetErrorString(e));
  double h = 0.0;
  for (double x : hd) h += x;
  const double g = c->gamma;
  *dgamma = h * (-2.0 / ((g - 1.0) * (g - 1.0)));  // D + K = 2/(gamma - 1)
  return FDLB_OK;
}

int fdlb_forward_ckpt(fdlb_ctx* c, int64_t nsteps, int every, void* ckpt) {
  if (!c || !ckpt || nsteps < 0 || every < 1) return fdlb::ctx_error(c, FDLB_EINVAL, "bad arguments");
  if (!adjoint_lattice(c))
    return fdlb::ctx_error(c, FDLB_EINVAL, "checkpointed runs: 1-D binary64 outlet contexts");
  int rc = fdlb::ctx_prepare(c);
  if (rc) return rc;
  const size_t bytes = fdlb_state_bytes(c);
  char* ck = (char*)ckpt;
  cudaError_t e = cudaSuccess;
  for (int64_t s = 0; s <= nsteps && e == cudaSuccess; ++s) {
    if (s % every == 0)
      e = cudaMemcpyAsync(ck + (s / every) * bytes, c->dp.F, bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (s == nsteps || e != cudaSuccess) break;
    for (int st : {fdlb::kStage3, fdlb::kStage4, fdlb::kFinal}) {
      int le = fdlb::ctx_launch_stage(c, st, c->stream);
      if (le) {
        e = (cudaError_t)le;
        break;
      }
    }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->status_host, c->dp.status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                        c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return fdlb::ctx_error(c, FDLB_ECUDA, cudaGetErrorString(e));
  if (*c->status_host & 1u)
    return fdlb::ctx_error(c, FDLB_EUNSTABLE, "a cell reached n <= 0, T <= 0 or a non-finite moment");
  return FDLB_OK;
}

int fdlb_adjoint(fdlb_ctx* c, int64_t nsteps, int every, const void* ckpt, double* Fbar,
                 double* dparams) {
  if (!c || !ckpt || !Fbar || !dparams || nsteps < 0 || every < 1)
    return fdlb::ctx_error(c, FDLB_EINVAL, "bad arguments");
  if (!adjoint_lattice(c))
    return fdlb::ctx_error(c, FDLB_EINVAL, "the adjoint covers 1-D binary64 outlet contexts");
  const size_t bytes = fdlb_state_bytes(c);
  // work space: two segment buffers, each holding per step of a segment the
  // saved F^n, F2, F3 and F4 (one more slot for the state after the
  // segment's last step); 5 adjoint arrays; the scalar accumulators
  const size_t seg_states = (size_t)(4 * every + 4);
  // the scalar accumulators: one row per block of the adjoint kernels
  const int64_t nblk = (c->dp.nx + fdlb::kTX - 1) / fdlb::kTX;
  const size_t scal_bytes = (size_t)nblk * fdlb::kNumAdjScalars * sizeof(double);
  const size_t need = (2 * seg_states + 5) * bytes + scal_bytes + 256;
  if (c->adj_bytes < need) {
    if (c->adj_buf) cudaFree(c->adj_buf);
    c->adj_buf = nullptr;
    c->adj_bytes = 0;
    cudaError_t e = cudaMalloc(&c->adj_buf, need);
    if (e != cudaSuccess) return fdlb::ctx_error(c, FDLB_ENOMEM, "adjoint work space");
    c->adj_bytes = need;
  }
  char* w = (char*)c->adj_buf;
  auto slot = [&](int buf, int64_t k, int which) {
    return (double*)(w + (buf * seg_states + (size_t)k * 4 + which) * bytes);
  };
  double* A4b = (double*)(w + 2 * seg_states * bytes);
  double* X3b = A4b + bytes / 8;
  double* X2b = X3b + bytes / 8;
  double* Fpt = X2b + bytes / 8;
  double* Db = Fpt + bytes / 8;
  double* scal = Db + bytes / 8;
  cudaStream_t s = c->stream;
  // The segments are processed last first.  Each segment's forward states are
  // recomputed from its checkpoint on a second stream, into the buffer the
  // adjoint of the segment after it no longer reads, while that adjoint runs:
  // both are chains of small launches that leave most of the GPU idle, so
  // they overlap.  Events order a segment's adjoint after its recompute, and
  // a buffer's recompute after the adjoint that last read it.
  cudaStream_t rs = nullptr;
  cudaEvent_t ev_start = nullptr, rdone[2] = {nullptr, nullptr}, adone[2] = {nullptr, nullptr};
  bool aused[2] = {false, false};
  cudaError_t e = cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&rdone[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&adone[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(scal, 0, scal_bytes, s);
  // the recompute stream starts after everything already queued on s
  if (e == cudaSuccess) e = cudaEventRecord(ev_start, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(rs, ev_start, 0);
  const int64_t nseg = (nsteps + every - 1) / every;
  for (int64_t sg = nseg - 1; sg >= 0 && e == cudaSuccess; --sg) {
    const int b = (int)(sg & 1);
    const int64_t s0 = sg * every;
    const int64_t ns = (nsteps - s0 < every) ? nsteps - s0 : every;
    // recompute the segment from its checkpoint: every launch gets its own
    // array pointers, so the stage kernels leave F^n, F2, F3 and F4 of each
    // step in its slot (the final stage writes F^{n+1} and its F2 into the
    // next slot); D and Af are the context's own scratch arrays, used by
    // the recomputes alone
    if (aused[b]) e = cudaStreamWaitEvent(rs, adone[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(slot(b, 0, 0), (const char*)ckpt + sg * bytes, bytes,
                          cudaMemcpyDeviceToDevice, rs);
    int le = 0;
    if (e == cudaSuccess) {
      DevParams q = c->dp;
      q.F = slot(b, 0, 0);
      q.F2 = slot(b, 0, 1);
      le = fdlb::launch_stage(q, fdlb::kPrep, rs);
    }
    for (int64_t k = 0; k < ns && e == cudaSuccess && !le; ++k) {
      DevParams q = c->dp;
      q.F = slot(b, k, 0);
      q.F2 = slot(b, k, 1);
      q.F3 = slot(b, k, 2);
      q.A4 = slot(b, k, 3);
      le = fdlb::launch_stage(q, fdlb::kStage3, rs);
      if (!le) le = fdlb::launch_stage(q, fdlb::kStage4, rs);
      q.F = slot(b, k + 1, 0);
      q.F2 = slot(b, k + 1, 1);
      if (!le) le = fdlb::launch_stage(q, fdlb::kFinal, rs);
    }
    if (le) e = (cudaError_t)le;
    if (e == cudaSuccess) e = cudaEventRecord(rdone[b], rs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, rdone[b], 0);
    // adjoint steps of the segment, last step first; Fbar is updated in
    // place (the stage-2 adjoint reads no adjoint of F^{n+1})
    for (int64_t k = ns - 1; k >= 0 && e == cudaSuccess; --k) {
      fdlb::AdjParams a{};
      a.Fn = slot(b, k, 0);
      a.F2s = slot(b, k, 1);
      a.F3s = slot(b, k, 2);
      a.F4s = slot(b, k, 3);
      a.Gbar = Fbar;
      a.A4bar = A4b;
      a.X3bar = X3b;
      a.X2bar = X2b;
      a.Fpart = Fpt;
      a.Dbar = Db;
      a.Gnew = Fbar;
      a.scal = scal;
      int r = launch_adj_any(4, c->dp, a, s);
      if (!r) r = launch_adj_any(3, c->dp, a, s);
      if (!r) r = launch_adj_any(2, c->dp, a, s);
      if (r) e = (cudaError_t)r;
    }
    if (e == cudaSuccess) e = cudaEventRecord(adone[b], s);
    aused[b] = true;
  }
  // s has waited for every recompute it used; let it also cover the stream's
  // tail before the stream goes away
  if (rs) {
    cudaEvent_t tail = nullptr;
    if (cudaEventCreateWithFlags(&tail, cudaEventDisableTiming) == cudaSuccess) {
      if (cudaEventRecord(tail, rs) == cudaSuccess) cudaStreamWaitEvent(s, tail, 0);
      cudaEventDestroy(tail);
    }
  }
  std::vector<double> rows((size_t)nblk * fdlb::kNumAdjScalars, 0.0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rows.data(), scal, scal_bytes, cudaMemcpyDeviceToHost, s);
  const cudaError_t es = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = es;
  // the blocks' rows summed in block order
  double h[fdlb::kNumAdjScalars] = {0};
  for (int64_t b = 0; b < nblk; ++b)
    for (int i = 0; i < fdlb::kNumAdjScalars; ++i) h[i] += rows[(size_t)b * fdlb::kNumAdjScalars + i];
  for (int i = 0; i < 2; ++i) {
    if (rdone[i]) cudaEventDestroy(rdone[i]);
    if (adone[i]) cudaEventDestroy(adone[i]);
  }
  if (ev_start) cudaEventDestroy(ev_start);
  if (rs) {
    cudaStreamSynchronize(rs);
    cudaStreamDestroy(rs);
  }
  if (e != cudaSuccess) return fdlb::ctx_error(c, FDLB_ECUDA, cudaGetErrorString(e));
  // the context's D and Af scratch arrays were overwritten: derive them anew
  c->prepared = false;
  // d/dgamma through D + K = 2/(gamma - 1); d/dtau through lam = dt/tau
  const double g = c->gamma;
  dparams[0] = h[fdlb::kBarDK] * (-2.0 / ((g - 1.0) * (g - 1.0)));
  const double lam = c->dt / c->tau;
  double dc[fdlb::kNumAdjScalars] = {0};
  stage_coef_dlam(lam, dc);
  double dlam = 0.0;
  for (int i = 0; i < fdlb::kBarDK; ++i) dlam += h[i] * dc[i];
  dparams[1] = dlam * (-lam / c->tau);
  return fdlb::ctx_prepare(c);
}

}  // extern "C"
