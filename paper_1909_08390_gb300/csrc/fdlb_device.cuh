// fdlb_device.cuh -- device helpers shared by the binary64 stage kernels
// (fdlb_kernels.cu), the binary32 stage kernels (fdlb_mixed.cu) and the
// adjoint: tile shapes, ghost indexing, the Hermite equilibrium factors
// (Eq. gExpanded), the moment sums (Eq. Moments_discrete) in binary64 and in
// compensated binary32 pairs, and the stage coefficients.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "fdlb_internal.h"
#include "fdlb_mp9.cuh"
#include "fdlb_tile.cuh"

namespace fdlb {
namespace {

constexpr int H = kGhost;  // ghost nodes per side (Sec. IV)

template <int DIM, int VAR = 0>
struct TileCfg;
// 2-D: 16 x 16 cells, 4 populations per group; 128 threads march the 4 x 32
// tile lines (16 along x, 16 along y) of a group, one line each.
template <>
struct TileCfg<2, 0> {
  static constexpr int TX = 16, TY = 16, NT = 128, G = 4, SEG = TX + 1;
};
// 1-D: 127 cells, 8 populations per group; 128 threads march 16 segments of
// 8 interfaces of each of the 8 lines.
template <>
struct TileCfg<1, 0> {
  static constexpr int TX = 127, TY = 1, NT = 128, G = 8, SEG = 8;
};
// 1-D: 63 cells, 16 populations per group, 8 segments of 8 interfaces.
template <>
struct TileCfg<1, 1> {
  static constexpr int TX = 63, TY = 1, NT = 128, G = 16, SEG = 8;
};
// 1-D: 255 cells, 8 populations per group, 16 segments of 16 interfaces.
template <>
struct TileCfg<1, 2> {
  static constexpr int TX = 255, TY = 1, NT = 128, G = 8, SEG = 16;
};
// 1-D: 15 and 31 cells, 16 populations per group, 64 threads: short single
// problems, so that their tiles still spread over the SMs.
template <>
struct TileCfg<1, 3> {
  static constexpr int TX = 15, TY = 1, NT = 64, G = 16, SEG = 4;
};
template <>
struct TileCfg<1, 4> {
  static constexpr int TX = 31, TY = 1, NT = 64, G = 16, SEG = 8;
};

// Tile shape of a single 1-D problem of nx cells: the largest tile that
// still gives about one tile per SM of GB300 (152), down to 15 cells.
inline int single_1d_variant(int64_t nx) {
  if (nx >= 127 * 152) return 0;
  if (nx >= 63 * 152) return 1;
  if (nx >= 31 * 152) return 4;
  return 3;
}
inline int tile_cells_1d(int variant) {
  switch (variant) {
    case 1: return TileCfg<1, 1>::TX;
    case 2: return TileCfg<1, 2>::TX;
    case 3: return TileCfg<1, 3>::TX;
    case 4: return TileCfg<1, 4>::TX;
    default: return TileCfg<1, 0>::TX;
  }
}

// Shared memory of one tile: the advected populations of a group on tile +
// halo, and the interface values along x and y.
template <int DIM, typename S, int VAR>
struct TileSmem {
  using C = TileCfg<DIM, VAR>;
  static constexpr int SX = C::TX + 2 * 5 + (DIM == 2 ? 1 : 0);  // padded row pitch (2-D)
  static constexpr int SY = DIM == 2 ? C::TY + 2 * 5 : 1;
  S tile[C::G][SY][SX];
  S hx[C::G][C::TY][C::TX + 1];
  S hy[DIM == 2 ? C::G : 1][DIM == 2 ? C::TX : 1][C::TY + 1];
};

// Where a tile lives: its problem's size, first cell in the population
// arrays, and gas and grid constants.
struct Geo {
  int nx, ny;
  int64_t base;
  double kchi, invDK, dtdx, dtdy;
  int prob;  // batch problem index, -1 for a single-problem context
};

// One axis of the Hermite-expanded equilibrium (Eq. gExpanded):
// g_k = sum_{l<Q} [w_k He_l(p_k)/l!] a_l(u, T) with
// a_l = sum_s l!/(2^s s!(l-2s)!) (T-1)^s u^(l-2s), generated by the
// recurrence a_0 = 1, a_1 = u, a_l = u a_{l-1} + (l-1)(T-1) a_{l-2}.
// The nodes are antisymmetric (p_{Q-1-k} = -p_k, so He_l(p_{Q-1-k}) =
// (-1)^l He_l(p_k)): g_k = E_k + O_k and g_{Q-1-k} = E_k - O_k with E/O the
// even/odd-l partial sums.
template <int Q>
__device__ __forceinline__ void axis_g(const double* wH, double u, double T, double (&g)[Q]) {
  double a[Q];
  a[0] = 1.0;
  if (Q > 1) a[1] = u;
  const double tm1 = T - 1.0;
#pragma unroll
  for (int l = 2; l < Q; ++l) a[l] = fma(u, a[l - 1], ((double)(l - 1) * tm1) * a[l - 2]);
#pragma unroll
  for (int k = 0; k < (Q + 1) / 2; ++k) {
    double e = wH[k];  // l = 0 (a_0 = 1)
    double o = 0.0;
#pragma unroll
    for (int l = 1; l < Q; ++l) {
      if (l & 1) o = fma(wH[l * kMaxQ + k], a[l], o);
      else e = fma(wH[l * kMaxQ + k], a[l], e);
    }
    g[k] = e + o;
    if (Q - 1 - k != k) g[Q - 1 - k] = e - o;
  }
}

template <int DIM, int QP, int QC>
struct Lat {
  static constexpr int NPHI = DIM == 1 ? QP : QP * QP;
  static constexpr int NCHI = DIM == 1 ? QC : QC * QC;
  static constexpr int P = NPHI + NCHI;
};

struct Moments {
  double n, jx, jy, e;
};

// phi: n += v, j += p v, e += p^2 v;  chi: e += v (Eq. Moments_discrete)
template <int DIM, int QP, int QC>
__device__ __forceinline__ void accumulate(const DevParams& p, Moments& m, int pop, double v) {
  using L = Lat<DIM, QP, QC>;
  if (pop < L::NPHI) {
    m.n += v;
    m.jx = fma(p.px[pop], v, m.jx);
    if (DIM == 2) m.jy = fma(p.py[pop], v, m.jy);
    m.e = fma(p.p2[pop], v, m.e);
  } else {
    m.e += v;
  }
}

// Per-cell equilibrium factors: feq(phi kx,ky) = hp[kx] * gyp[ky],
// feq(chi qx,qy) = hc[qx] * gyc[qy] (1-D: hp[kx], hc[qx]).
template <int DIM, int QP, int QC>
struct EqCell {
  double hp[QP], gyp[DIM == 2 ? QP : 1];
  double hc[QC], gyc[DIM == 2 ? QC : 1];
};

// Factors from (n, u, T); phi^eq = n prod g, chi^eq = (D+K-d) T n prod g^chi.
template <int DIM, int QP, int QC>
__device__ __forceinline__ void make_eq_nut(const DevParams& p, double kchi, double n, double ux,
                                            double uy, double T, EqCell<DIM, QP, QC>& eq) {
  double gx[QP];
  axis_g<QP>(p.wHp, ux, T, gx);
#pragma unroll
  for (int k = 0; k < QP; ++k) eq.hp[k] = n * gx[k];
  if constexpr (DIM == 2) axis_g<QP>(p.wHp, uy, T, eq.gyp);
  const double nchi = kchi * T * n;
  if constexpr (QC == QP) {
#pragma unroll
    for (int k = 0; k < QC; ++k) eq.hc[k] = nchi * gx[k];
    if constexpr (DIM == 2) {
#pragma unroll
      for (int k = 0; k < QC; ++k) eq.gyc[k] = eq.gyp[k];
    }
  } else {
    double gc[QC];
    axis_g<QC>(p.wHc, ux, T, gc);
#pragma unroll
    for (int k = 0; k < QC; ++k) eq.hc[k] = nchi * gc[k];
    if constexpr (DIM == 2) axis_g<QC>(p.wHc, uy, T, eq.gyc);
  }
}

// n, u and T = (sum phi p^2 + sum chi - n u^2) / ((D+K) n) from the moment
// sums; false if the cell is not a valid gas state.
template <int DIM>
__device__ __forceinline__ bool moments_to_nut(double invDK, const Moments& m, double& n,
                                               double& ux, double& uy, double& T) {
  n = m.n;
  const double inv_n = 1.0 / n;
  ux = m.jx * inv_n;
  uy = DIM == 2 ? m.jy * inv_n : 0.0;
  T = (m.e - n * fma(ux, ux, uy * uy)) * inv_n * invDK;
  return (n > 0.0) && (T > 0.0) && isfinite(n) && isfinite(T) && isfinite(ux) && isfinite(uy);
}

// ---- storage-type helpers --------------------------------------------------

__device__ __forceinline__ double sfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float sfma(float a, float b, float c) { return fmaf(a, b, c); }

// Moment sums of binary32 populations, kept as unevaluated binary32 pairs
// (hi + lo) with error-free transformations: TwoSum for each addition and the
// fma-exact product error for p * v with p = hi + lo split on the host.  The
// pairs carry about 44 significant bits, so n, u and T = (E - n u^2)/((D+K) n)
// are recovered without the cancellation's loss although the populations are
// binary32: the stage kernels go on in pair arithmetic (fdlb_mixed.cu), the
// moments output folds the pairs into binary64 once per cell.
struct MomentsF {
  float nh, nl, jxh, jxl, jyh, jyl, eh, el;
};

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

__device__ __forceinline__ void two_prod_acc(float& hi, float& lo, float ph, float pl, float v) {
  const float prod = __fmul_rn(ph, v);
  const float perr = fmaf(ph, v, -prod);  // exact: ph * v - prod
  two_sum_acc(hi, lo, prod);
  lo = __fadd_rn(lo, fmaf(pl, v, perr));
}

template <int DIM, int QP, int QC>
__device__ __forceinline__ void accumulate(const DevParams& p, MomentsF& m, int pop, float v) {
  using L = Lat<DIM, QP, QC>;
  if (pop < L::NPHI) {
    two_sum_acc(m.nh, m.nl, v);
    two_prod_acc(m.jxh, m.jxl, p.pxh[pop], p.pxl[pop], v);
    if (DIM == 2) two_prod_acc(m.jyh, m.jyl, p.pyh[pop], p.pyl[pop], v);
    two_prod_acc(m.eh, m.el, p.p2h[pop], p.p2l[pop], v);
  } else {
    two_sum_acc(m.eh, m.el, v);
  }
}

// The same sums for two cells at once, in packed binary32 pairs (sm_100 and
// later: one instruction per two lanes).  Each lane performs exactly the
// operations of the scalar version, so the sums are bitwise the same.
struct MomentsF2 {
  float2 nh, nl, jxh, jxl, jyh, jyl, eh, el;
};
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, f2s(-1.0f), a);  // a - b, rounded once
}
__device__ __forceinline__ void two_sum_acc2(float2& hi, float2& lo, float2 x) {
  const float2 s = __fadd2_rn(hi, x);
  const float2 bb = sub2(s, hi);
  const float2 err = __fadd2_rn(sub2(hi, sub2(s, bb)), sub2(x, bb));
  hi = s;
  lo = __fadd2_rn(lo, err);
}
__device__ __forceinline__ void two_prod_acc2(float2& hi, float2& lo, float ph, float pl,
                                              float2 v) {
  const float2 prod = __fmul2_rn(f2s(ph), v);
  const float2 nprod = __fmul2_rn(f2s(-ph), v);   // -prod exactly
  const float2 perr = __ffma2_rn(f2s(ph), v, nprod);  // exact: ph * v - prod
  two_sum_acc2(hi, lo, prod);
  lo = __fadd2_rn(lo, __ffma2_rn(f2s(pl), v, perr));
}
template <int DIM, int QP, int QC>
__device__ __forceinline__ void accumulate2(const DevParams& p, MomentsF2& m, int pop, float2 v) {
  using L = Lat<DIM, QP, QC>;
  if (pop < L::NPHI) {
    two_sum_acc2(m.nh, m.nl, v);
    two_prod_acc2(m.jxh, m.jxl, p.pxh[pop], p.pxl[pop], v);
    if (DIM == 2) two_prod_acc2(m.jyh, m.jyl, p.pyh[pop], p.pyl[pop], v);
    two_prod_acc2(m.eh, m.el, p.p2h[pop], p.p2l[pop], v);
  } else {
    two_sum_acc2(m.eh, m.el, v);
  }
}
// lane i (0 or 1) of a pair of sums
__device__ __forceinline__ MomentsF lane(const MomentsF2& m, int i) {
  auto g = [i](float2 x) { return i == 0 ? x.x : x.y; };
  return MomentsF{g(m.nh), g(m.nl), g(m.jxh), g(m.jxl), g(m.jyh), g(m.jyl), g(m.eh), g(m.el)};
}

__device__ __forceinline__ Moments to_fp64(const Moments& m) { return m; }
__device__ __forceinline__ Moments to_fp64(const MomentsF& m) {
  return Moments{(double)m.nh + (double)m.nl, (double)m.jxh + (double)m.jxl,
                 (double)m.jyh + (double)m.jyl, (double)m.eh + (double)m.el};
}

template <typename S>
struct MomAcc;
template <>
struct MomAcc<double> {
  using type = Moments;
};
template <>
struct MomAcc<float> {
  using type = MomentsF;
};

// Equilibrium factors in the storage type (binary32 copies of the binary64
// per-cell factors on the mixed path).
template <int DIM, int QP, int QC, typename S>
struct EqCellS {
  S hp[QP], gyp[DIM == 2 ? QP : 1];
  S hc[QC], gyc[DIM == 2 ? QC : 1];
};

template <int DIM, int QP, int QC, typename S>
__device__ __forceinline__ void to_storage(const EqCell<DIM, QP, QC>& a, EqCellS<DIM, QP, QC, S>& b) {
#pragma unroll
  for (int k = 0; k < QP; ++k) b.hp[k] = (S)a.hp[k];
#pragma unroll
  for (int k = 0; k < QC; ++k) b.hc[k] = (S)a.hc[k];
  if constexpr (DIM == 2) {
#pragma unroll
    for (int k = 0; k < QP; ++k) b.gyp[k] = (S)a.gyp[k];
#pragma unroll
    for (int k = 0; k < QC; ++k) b.gyc[k] = (S)a.gyc[k];
  }
}

template <int DIM, int QP, int QC, typename S>
__device__ __forceinline__ S feq_of(const EqCellS<DIM, QP, QC, S>& eq, int pop) {
  using L = Lat<DIM, QP, QC>;
  if (pop < L::NPHI) {
    if constexpr (DIM == 1) return eq.hp[pop];
    else return eq.hp[pop % QP] * eq.gyp[pop / QP];
  }
  const int q = pop - L::NPHI;
  if constexpr (DIM == 1) return eq.hc[q];
  else return eq.hc[q % QC] * eq.gyc[q / QC];
}

// Stage coefficients in the storage type (computed in binary64 on the host).
template <typename S>
struct CoefS {
  S k3, k4, kf, at32, at42, at43, wt2, wt3, wt4, a33e3, a43e3, w3e3, a44e4, w4e4, c2;
  __device__ __forceinline__ explicit CoefS(const StageCoef& c)
      : k3((S)c.k3), k4((S)c.k4), kf((S)c.kf), at32((S)c.at32), at42((S)c.at42),
        at43((S)c.at43), wt2((S)c.wt2), wt3((S)c.wt3), wt4((S)c.wt4), a33e3((S)c.a33e3),
        a43e3((S)c.a43e3), w3e3((S)c.w3e3), a44e4((S)c.a44e4), w4e4((S)c.w4e4), c2((S)c.c2) {}
};

// Asynchronous global -> shared copies of one element (4 or 8 bytes): the
// prefetch of the next population group.  A thread that copies elements
// waits on its own copies before reading them, or before a barrier after
// which other threads read them.
template <typename S>
__device__ __forceinline__ void cp_async(S* smem, const S* gmem) {
  static_assert(sizeof(S) == 4 || sizeof(S) == 8, "4- or 8-byte elements");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(S) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
// all but the most recently committed group complete
__device__ __forceinline__ void cp_async_wait_1() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

// Lattices of the batch kernels (1-D).
#define FDLB_BATCH_LATTICES(X) \
  X(8, 8)                      \
  X(5, 3)

// Dispatch over the compiled (d, Qphi, Qchi) instances.
#define FDLB_LATTICES(X) \
  X(1, 8, 8)             \
  X(2, 8, 8)             \
  X(1, 5, 3)             \
  X(2, 5, 3)             \
  X(1, 3, 3)             \
  X(2, 3, 3)

}  // namespace
}  // namespace fdlb
