// fdlb_mixed.cu -- binary32 stage kernels of the IMEX step (FDLB_MIXED):
// one pass over memory per advected stage.
//
// Storage.  Every population of the state F^n is an unevaluated pair of
// binary32 values sh + sl with |sl| <= ulp(sh)/2 (about 48 significant
// bits).  The explicit parts of the stages are kept as binary32 low parts
// relative to sh (R3 = sh + r3l, A4' = sh + a4l, A_fin = sh + afl), which are
// small where the flow is smooth, so their rounding is relative to the
// increment and not to the population.  A binary32 copy of F rounded at each
// stage loses about 6e-8 of every population per stage; over thousands of
// steps that noise moves shocks and contacts by far more than the 1e-5 the
// mixed path is held to.
//
// Each kernel relaxes the previous stage while it stages its advected
// values (Sec. III closed forms), from per-cell records of the previous
// stage's equilibrium factors (Eq. gExpanded, evaluated in binary32-pair
// arithmetic and kept as pairs):
//   stage 3 stages F2 = E0 + c2 D with D = F^n - E0,
//   stage 4 stages F3 = R3 - a33 e3 D3 with D3 = R3 - E3,
//   the final stage stages F4 = R4 - a44 e4 D4 with D4 = R4 - E4,
// every D formed as (sh - Eh) + (low part - El), accurate to its own size.
// On 2-D tiles the staged values are taken relative to one value per
// population and tile (the state's sh at the tile's first cell): the MP-9
// march is translation invariant, and the shift keeps its binary32 rounding
// relative to the variation across the tile instead of to the populations.
//
// Moments (Eq. Moments_discrete) of R3 and R4 are the binary64 per-cell sums
// of sh (mhi, from the previous final stage) plus binary32 sums of the low
// parts; the final stage sums the new state's sh with error-free
// transformations (TwoSum and the fma product error) and its sl plainly.
// n, u and T (the cancellation T = (e - j u)/((D+K) n) included) are then
// recovered in binary64, and the record of the next equilibrium is written.
//
// Arrays per population and step: stage 3 reads sh, sl and writes r3l, a4l,
// afl; stage 4 reads sh, r3l, a4l, afl and writes a4l (now R4's low part)
// and afl; the final stage reads sh, a4l, afl and writes the new nh, nl --
// 16 binary32 accesses, plus the records and mhi per cell.
#include "fdlb_device.cuh"

namespace fdlb {
namespace {

// Components of a cell's record.  phi^eq(kx, ky) = A[kx] * B[ky] with
// A = n g_x, B = g_y (1-D: A[k]); chi^eq(qx, qy) = C * A[qx] * B[qy] with
// C = (D+K-d) T when Qchi = Qphi, else Hx[qx] * Hy[qy] with Hx = nchi h_x.
// 2-D records with Qchi = Qphi also hold CB[ky] = C B[ky], so that
// chi^eq = A[qx] * CB[qy] takes the same two factors as phi^eq.  Every
// component is a binary32 pair: high parts at components 0..W-1, low parts
// at W..2W-1.
template <int DIM, int QP, int QC>
struct RecLayout {
  static constexpr bool kSame = QP == QC;
  static constexpr int kChi = DIM == 1 ? QP : 2 * QP;  // first chi component
  static constexpr bool kCB = DIM == 2 && kSame;
  static constexpr int kCBo = kChi + 1;               // first CB component
  static constexpr int W = kSame ? kChi + 1 + (kCB ? QP : 0) : kChi + (DIM == 1 ? QC : 2 * QC);
  static_assert(!kCB || kCBo + QP == W, "CB components close the record");
};

// ---- binary32 pairs: x = hi + lo with about 48 significant bits ----------
// The classical error-free arithmetic (Dekker, Knuth): TwoSum for additions,
// the fused multiply-add for the exact product error; the intrinsics keep
// the compiler from contracting the error terms away.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_quick(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
  const float s = __fadd_rn(x.hi, y.hi);
  const float bb = __fsub_rn(s, x.hi);
  const float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));
  return df_quick(s, __fadd_rn(e, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ DF df_neg(DF x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  const float pr = __fmul_rn(x.hi, y.hi);
  float e = fmaf(x.hi, y.hi, -pr);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return df_quick(pr, e);
}
__device__ __forceinline__ DF df_of(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

// The same pair arithmetic on two lanes at once (packed binary32, sm_100
// and later); each lane performs exactly the operations of DF.
struct DF2 {
  float2 hi, lo;
};
__device__ __forceinline__ float2 neg2(float2 x) { return __fmul2_rn(x, f2s(-1.0f)); }
__device__ __forceinline__ DF2 df_quick2(float2 a, float2 b) {
  const float2 s = __fadd2_rn(a, b);
  return {s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ DF2 df_add2(DF2 x, DF2 y) {
  const float2 s = __fadd2_rn(x.hi, y.hi);
  const float2 bb = sub2(s, x.hi);
  const float2 e = __fadd2_rn(sub2(x.hi, sub2(s, bb)), sub2(y.hi, bb));
  return df_quick2(s, __fadd2_rn(e, __fadd2_rn(x.lo, y.lo)));
}
__device__ __forceinline__ DF2 df_mul2(DF2 x, DF2 y) {
  const float2 pr = __fmul2_rn(x.hi, y.hi);
  float2 e = __ffma2_rn(x.hi, y.hi, neg2(pr));
  e = __ffma2_rn(x.hi, y.lo, e);
  e = __ffma2_rn(x.lo, y.hi, e);
  return df_quick2(pr, e);
}
__device__ __forceinline__ DF2 df_bcast(DF x) { return {f2s(x.hi), f2s(x.lo)}; }

// Product of two pairs without renormalising (hi = x.hi y.hi rounded, lo the
// rest to binary32 accuracy): an equilibrium population from its factors.
__device__ __forceinline__ DF pmul(DF x, DF y) {
  const float h = __fmul_rn(x.hi, y.hi);
  float l = fmaf(x.hi, y.hi, -h);
  l = fmaf(x.hi, y.lo, l);
  l = fmaf(x.lo, y.hi, l);
  return {h, l};
}
__device__ __forceinline__ DF2 pmul2(DF2 x, DF2 y) {
  const float2 h = __fmul2_rn(x.hi, y.hi);
  float2 l = __ffma2_rn(x.hi, y.hi, neg2(h));
  l = __ffma2_rn(x.hi, y.lo, l);
  l = __ffma2_rn(x.lo, y.hi, l);
  return {h, l};
}

// One axis of the equilibrium factors (Eq. gExpanded) times `scale`, in pair
// arithmetic: the recurrence a_0 = s, a_1 = s u, a_l = u a_{l-1} +
// (l-1)(T-1) a_{l-2}, then g_k = sum_l [w_k He_l(p_k)/l!] a_l, summed as even
// and odd parts over the antisymmetric nodes like axis_g.
template <int Q>
__device__ __forceinline__ void axis_g_df(const float* ch, const float* cl, DF u, DF T, DF scale,
                                          DF (&g)[Q]) {
  DF a[Q];
  a[0] = scale;
  if (Q > 1) a[1] = df_mul(scale, u);
  const DF tm1 = df_add(T, DF{-1.0f, 0.0f});
#pragma unroll
  for (int l = 2; l < Q; ++l)
    a[l] = df_add(df_mul(u, a[l - 1]), df_mul(df_mul(DF{(float)(l - 1), 0.0f}, tm1), a[l - 2]));
  // nodes k and k+1 in the two lanes of packed pairs, then an odd one out
  constexpr int NH = (Q + 1) / 2;
#pragma unroll
  for (int k = 0; k + 1 < NH; k += 2) {
    auto coef = [&](int l) {
      return DF2{make_float2(ch[l * kMaxQ + k], ch[l * kMaxQ + k + 1]),
                 make_float2(cl[l * kMaxQ + k], cl[l * kMaxQ + k + 1])};
    };
    DF2 e = df_mul2(coef(0), df_bcast(a[0]));
    DF2 o = DF2{f2s(0.0f), f2s(0.0f)};
#pragma unroll
    for (int l = 1; l < Q; ++l) {
      const DF2 t = df_mul2(coef(l), df_bcast(a[l]));
      if (l & 1) o = df_add2(o, t);
      else e = df_add2(e, t);
    }
    const DF2 sum = df_add2(e, o);
    const DF2 dif = df_add2(e, DF2{neg2(o.hi), neg2(o.lo)});
    g[k] = DF{sum.hi.x, sum.lo.x};
    if (Q - 1 - k != k) g[Q - 1 - k] = DF{dif.hi.x, dif.lo.x};
    g[k + 1] = DF{sum.hi.y, sum.lo.y};
    if (Q - 2 - k != k + 1) g[Q - 2 - k] = DF{dif.hi.y, dif.lo.y};
  }
  if constexpr (NH % 2 == 1) {
    constexpr int k = NH - 1;
    DF e = df_mul(DF{ch[k], cl[k]}, a[0]);
    DF o = DF{0.0f, 0.0f};
#pragma unroll
    for (int l = 1; l < Q; ++l) {
      const DF t = df_mul(DF{ch[l * kMaxQ + k], cl[l * kMaxQ + k]}, a[l]);
      if (l & 1) o = df_add(o, t);
      else e = df_add(e, t);
    }
    g[k] = df_add(e, o);
    if (Q - 1 - k != k) g[Q - 1 - k] = df_add(e, df_neg(o));
  }
}

// Record of the equilibrium of (n, u, T) at cell `cell` of rec (components N
// apart, high parts then low parts), in pair arithmetic.
template <int DIM, int QP, int QC>
__device__ __forceinline__ void write_record(const DevParams& p, DF kchi, DF n, DF ux, DF uy, DF T,
                                             float* __restrict__ rec, int64_t cell, int64_t N) {
  using R = RecLayout<DIM, QP, QC>;
  constexpr int W = R::W;
  auto put = [&](int k, DF v) {
    rec[k * N + cell] = v.hi;
    rec[(W + k) * N + cell] = v.lo;
  };
  const DF one{1.0f, 0.0f};
  DF g[QP];
  axis_g_df<QP>(p.wHph, p.wHpl, ux, T, n, g);
#pragma unroll
  for (int k = 0; k < QP; ++k) put(k, g[k]);
  if constexpr (DIM == 2) {
    axis_g_df<QP>(p.wHph, p.wHpl, uy, T, one, g);
#pragma unroll
    for (int k = 0; k < QP; ++k) put(QP + k, g[k]);
  }
  const DF kT = df_mul(kchi, T);
  if constexpr (R::kSame) {
    put(R::kChi, kT);
    if constexpr (R::kCB) {  // g holds the y factors B
#pragma unroll
      for (int k = 0; k < QP; ++k) put(R::kCBo + k, df_mul(kT, g[k]));
    }
  } else {
    DF h[QC];
    axis_g_df<QC>(p.wHch, p.wHcl, ux, T, df_mul(kT, n), h);
#pragma unroll
    for (int q = 0; q < QC; ++q) put(R::kChi + q, h[q]);
    if constexpr (DIM == 2) {
      axis_g_df<QC>(p.wHch, p.wHcl, uy, T, one, h);
#pragma unroll
      for (int q = 0; q < QC; ++q) put(R::kChi + QC + q, h[q]);
    }
  }
}

// Moment sums (n, jx, jy, e) of a cell, binary64 -> validity flags and the
// record of its equilibrium: u = j/n and T = (e - j.u)/((D+K) n) (Eq.
// Moments_discrete and the temperature definition) in binary64, the Hermite
// factors in pair arithmetic from the binary64 n, u, T.
template <int DIM, int QP, int QC>
__device__ __forceinline__ void finish_cell(const DevParams& p, double kchi, double invDK, int prob,
                                            double n, double jx, double jy, double e,
                                            float* __restrict__ rec, int64_t cell) {
  const double inv_n = 1.0 / n;
  const double ux = jx * inv_n;
  const double uy = DIM == 2 ? jy * inv_n : 0.0;
  const double T = (e - fma(jx, ux, jy * uy)) * inv_n * invDK;
  const bool ok = n > 0.0 && T > 0.0 && isfinite(n) && isfinite(T) && isfinite(ux) && isfinite(uy);
  if (!ok) {
    atomicOr(p.status, 1u);
    if (prob >= 0) atomicOr(&p.pstatus[prob], 1u);
  }
  write_record<DIM, QP, QC>(p, df_of(kchi), df_of(n), df_of(ux), df_of(uy), df_of(T), rec, cell,
                            p.N);
}

// Equilibrium pair of population pop from a record whose components lie
// `stride` floats apart (read through the read-only data cache).
template <int DIM, int QP, int QC>
__device__ __forceinline__ DF eq_from_rec(const float* __restrict__ rec, int64_t stride, int pop) {
  using R = RecLayout<DIM, QP, QC>;
  using L = Lat<DIM, QP, QC>;
  auto c = [&](int k) { return DF{rec[k * stride], rec[(R::W + k) * stride]}; };
  if (pop < L::NPHI) {
    if constexpr (DIM == 1) return c(pop);
    else return pmul(c(pop % QP), c(QP + pop / QP));
  }
  const int q = pop - L::NPHI;
  if constexpr (R::kSame) {
    if constexpr (DIM == 1) return pmul(c(R::kChi), c(q));
    else return pmul(c(q % QP), c(R::kCBo + q / QP));
  } else {
    if constexpr (DIM == 1) return c(R::kChi + q);
    else return pmul(c(R::kChi + q % QC), c(R::kChi + QC + q / QC));
  }
}

// Record prefetch plan of a population group, for lattices with Qchi = Qphi
// whose groups align with rows of the velocity grid ((8, 8) with groups of 4
// in 2-D; groups of 8 or 16 in 1-D).  Slot s of the group's buffer holds one
// record component (its high and low parts): slots 0..NA-1 the x factors A
// of the group's columns, then slot kB the second factor: in 2-D B of the
// group's row (phi) or CB (chi), in 1-D the chi factor C.
template <int DIM, int QP, int QC, int G>
struct GroupRec {
  static constexpr bool kOn =
      QP == QC && (DIM == 2 ? (QP % G == 0) : (QP % G == 0 || G % QP == 0));
  static constexpr int NA = G < QP ? G : QP;
  static constexpr int kB = NA;
  static constexpr int NS = kB + 1;
  // first x-factor component of group g0 (1-D groups of 2 QP start at 0)
  __device__ static int a0(int g0) {
    const int nphi = DIM == 2 ? QP * QP : QP;
    const int k0 = g0 >= nphi ? g0 - nphi : g0;
    return G > QP ? 0 : k0 % QP;
  }
  __device__ static bool has_chi(int g0) { return g0 + G > (DIM == 2 ? QP * QP : QP); }
  // record component held by slot s for group g0 (-1: unused)
  __device__ static int comp(int g0, int s) {
    const int nphi = DIM == 2 ? QP * QP : QP;
    using R = RecLayout<DIM, QP, QC>;
    if (s < NA) return a0(g0) + s;
    if (DIM == 2) return (g0 >= nphi ? R::kCBo + (g0 - nphi) / QP : QP + g0 / QP);
    return has_chi(g0) ? R::kChi : -1;
  }
};

// First population of group gi.  2-D groups with a record plan run
// x-block-major: the 8 groups that share the x factors A of one block of G
// columns come one after another (rows ky = 0..QP-1), phi before chi, so that
// only B (and C once) change from one group to the next.  Otherwise groups
// run in population order.  The final stage and the prep kernel sum the
// moments in this order, so that both give the same bits.
template <int DIM, int QP, int QC, int G>
__device__ __forceinline__ int group_pop(int gi) {
  using L = Lat<DIM, QP, QC>;
  if constexpr (DIM == 2 && GroupRec<DIM, QP, QC, G>::kOn) {
    constexpr int per_half = L::NPHI / G;
    const int half = gi / per_half, r = gi % per_half;
    return half * L::NPHI + (r % QP) * QP + (r / QP) * G;
  } else {
    return gi * G;
  }
}

template <int DIM, int QP, int QC, int VAR, int STAGE>
struct MixSmem {
  using C = TileCfg<DIM, VAR>;
  using GR = GroupRec<DIM, QP, QC, C::G>;
  static constexpr int SXH = C::TX + 2 * H;             // staged columns
  static constexpr int SX = SXH + (DIM == 2 ? 1 : 0);   // tile row pitch
  static constexpr int SY = DIM == 2 ? C::TY + 2 * H : 1;
  // staged cells: tile + halo without the 2-D corner blocks, which feed no
  // line (rows 0..H-1 and H+TY.. take the tile's columns only)
  static constexpr int NSC = DIM == 2 ? C::TY * SXH + 2 * H * C::TX : SXH;
  static constexpr int NSL = GR::kOn ? GR::NS : 1;
  float rawh[C::G][NSC];               // the state's high parts sh, as loaded
  float rawl[C::G][NSC];               // the advected array's low parts, as loaded
  float rbh[NSL][GR::kOn ? NSC : 1];   // the group's record components (GroupRec
  float rbl[NSL][GR::kOn ? NSC : 1];   // plan): high and low parts, as loaded
  float tile[C::G][SY][SX];            // relaxed advected populations - ref
  // 2-D: flux differences of the cells along x and y (mp9_march_delta_fp32);
  // 1-D: interface values along x.  Rows of TX + 1 (TY + 1) floats: the odd
  // pitch keeps the march's column-wise writes free of bank conflicts.
  float hx[C::G][C::TY][C::TX + 1];
  float hy[DIM == 2 ? C::G : 1][DIM == 2 ? C::TX : 1][DIM == 2 ? C::TY + 1 : 1];
  float ownd[C::G][C::TY * C::TX];     // R - F_eq of the own cells
  // stage 3: sl of the own cells; final stage: sh of the own cells
  float ownv[STAGE == kStage4 ? 1 : C::G][STAGE == kStage4 ? 1 : C::TY * C::TX];
  // dt p / ds per population as binary32 pairs: (x hi, x lo, y hi, y lo)
  float4 coef[Lat<DIM, QP, QC>::P];
};

// Plain binary32 moment sums of low parts (stages 3 and 4), two cells.
struct MomL2 {
  float2 n, jx, jy, e;
};
template <int DIM, int QP, int QC>
__device__ __forceinline__ void accum_low2(const DevParams& p, MomL2& m, int pop, float2 v) {
  using L = Lat<DIM, QP, QC>;
  if (pop < L::NPHI) {
    m.n = __fadd2_rn(m.n, v);
    m.jx = __ffma2_rn(f2s(p.pxh[pop]), v, m.jx);
    if (DIM == 2) m.jy = __ffma2_rn(f2s(p.pyh[pop]), v, m.jy);
    m.e = __ffma2_rn(f2s(p.p2h[pop]), v, m.e);
  } else {
    m.e = __fadd2_rn(m.e, v);
  }
}
struct MomL {
  float n, jx, jy, e;
};
template <int DIM, int QP, int QC>
__device__ __forceinline__ void accum_low(const DevParams& p, MomL& m, int pop, float v) {
  using L = Lat<DIM, QP, QC>;
  if (pop < L::NPHI) {
    m.n = __fadd_rn(m.n, v);
    m.jx = fmaf(p.pxh[pop], v, m.jx);
    if (DIM == 2) m.jy = fmaf(p.pyh[pop], v, m.jy);
    m.e = fmaf(p.p2h[pop], v, m.e);
  } else {
    m.e = __fadd_rn(m.e, v);
  }
}

// One tile of one stage.  Ends with every thread past its last use of the
// shared memory, so a persistent CTA may start its next tile at once.
template <int DIM, int QP, int QC, int STAGE, int VAR>
__device__ __forceinline__ void mixed_tile(const DevParams& p, const Geo& geo, int x0, int y0,
                                           MixSmem<DIM, QP, QC, VAR, STAGE>& sm) {
  using C = TileCfg<DIM, VAR>;
  using L = Lat<DIM, QP, QC>;
  using M = MixSmem<DIM, QP, QC, VAR, STAGE>;
  using R = RecLayout<DIM, QP, QC>;
  constexpr int TX = C::TX, TY = C::TY, NT = C::NT, G = C::G, SEG = C::SEG;
  constexpr int SX = M::SX, SXH = M::SXH, NSC = M::NSC;
  constexpr int CELLS = TX * TY;
  constexpr int CPT = (CELLS + NT - 1) / NT;
  constexpr int NSEG = (TX + 1) / SEG;
  static_assert(NSEG * SEG == TX + 1, "segments tile the line");
  constexpr int NLINE = DIM == 2 ? TX + TY : 1;
  static_assert(G * NLINE * NSEG == NT, "one march task per thread");
  constexpr int J = (NSC + NT - 1) / NT;  // staged cells per thread
  constexpr int W = R::W;

  const float* __restrict__ const Sh = p.sh;
  // the advected array's low parts: sl (stage 3), r3l (stage 4), a4l = R4's
  // low part (final stage)
  const float* __restrict__ const adv_l =
      STAGE == kStage3 ? p.sl : (STAGE == kStage4 ? p.r3l : p.a4l);
  const float* __restrict__ const rin =
      p.erec[STAGE == kStage3 ? 0 : (STAGE == kStage4 ? 1 : 2)];
  float* __restrict__ const rout = p.erec[STAGE == kStage3 ? 1 : (STAGE == kStage4 ? 2 : 0)];
  const int tid = threadIdx.x;
  const int64_t N = p.N;

  // this thread's staged cells: tile offset, cell offset from geo.base
  // (-1: none), own-cell index (-1: halo)
  int soff[J], goff[J], oidx[J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int e = tid + j * NT;
    // staged cell e (NSC of them), in the compact order of staged_pos
    int r, c;
    staged_pos(e, DIM, TX, TY, r, c);
    soff[j] = r * SX + c;
    goff[j] = -1;
    oidx[j] = -1;
    if (e < NSC) {
      const int gx = wrap_or_clamp(x0 - H + c, geo.nx, p.bc);
      const int gy = DIM == 2 ? wrap_or_clamp(y0 - H + r, geo.ny, p.bc) : 0;
      goff[j] = gy * geo.nx + gx;
      const int lx = c - H, ly = DIM == 2 ? r - H : 0;
      if (lx >= 0 && lx < TX && ly >= 0 && ly < TY && x0 + lx < geo.nx && y0 + ly < geo.ny)
        oidx[j] = ly * TX + lx;
    }
  }
  // own cells of this thread (pass 1)
  int lxs[CPT], lys[CPT];
  int64_t cell[CPT];
  bool valid[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    // a thread's cells are CPT consecutive ones (x-adjacent pairs when CPT =
    // 2 and TX is even), so that pass 1 can move them as 8-byte pairs; a
    // slot past the tile's cells takes cell 0's indices (its lane computes
    // on them and stores nothing), so every shared-memory index stays inside
    // its array
    const int ci = CPT * tid + k;
    const int c = ci < CELLS ? ci : 0;
    lxs[k] = c % TX;
    lys[k] = c / TX;
    valid[k] = (ci < CELLS) && (x0 + lxs[k] < geo.nx) && (y0 + lys[k] < geo.ny);
    cell[k] = geo.base + (int64_t)(y0 + lys[k]) * geo.nx + (x0 + lxs[k]);
  }
  // both cells of the pair valid, adjacent in memory and 8-byte aligned
  const bool pair_vec = CPT == 2 && valid[0] && valid[CPT - 1] &&
                        cell[CPT - 1] == cell[0] + 1 && (cell[0] & 1) == 0 && (N & 1) == 0;
  // moment sums: stages 3 and 4 sum the low parts plainly; the final stage
  // sums the new high parts error-free (mom*) and the new low parts plainly
  MomL lm[CPT];
  MomentsF mom[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    lm[k] = {};
    mom[k] = {};
  }
  MomL2 lm2 = {};
  MomentsF2 mom2 = {};
  const CoefS<float> sc(p.sc);
  const float arelax = STAGE == kStage3 ? sc.c2 : (STAGE == kStage4 ? sc.a33e3 : sc.a44e4);
  // coefficients that multiply advection terms of the size of the
  // populations' variation, as binary32 pairs: dt p / ds (a rounded speed
  // would shift every wave coherently) and the explicit weights wt2, wt3,
  // wt4 (1/6, 1/6, 2/3, whose rounded sum misses 1)
  const DF dtdx_df = df_of(geo.dtdx), dtdy_df = df_of(geo.dtdy);
  const float wtl = STAGE == kStage3 ? (float)(p.sc.wt2 - (double)sc.wt2)
                  : STAGE == kStage4 ? (float)(p.sc.wt3 - (double)sc.wt3)
                                     : (float)(p.sc.wt4 - (double)sc.wt4);
  // dt p / ds of every population along x and y as pairs, once per tile (the
  // first barrier of the group loop orders it before pass 1); 2-D takes |.|
  // (the flux differences of the 2-D march carry the velocity's sign)
  for (int pop = tid; pop < L::P; pop += NT) {
    DF cx = df_mul(dtdx_df, DF{p.pxh[pop], p.pxl[pop]});
    DF cy = DIM == 2 ? df_mul(dtdy_df, DF{p.pyh[pop], p.pyl[pop]}) : DF{0.0f, 0.0f};
    if (DIM == 2 && cx.hi < 0.0f) cx = df_neg(cx);
    if (DIM == 2 && cy.hi < 0.0f) cy = df_neg(cy);
    sm.coef[pop] = make_float4(cx.hi, cx.lo, cy.hi, cy.lo);
  }
  const float* __restrict__ const rbase = rin + geo.base;
  // the reference value of each population on a 2-D tile: sh at the tile's
  // first cell.  1-D tiles take none, so that a 1-D problem gives the same
  // bits whatever its tiling (batches and single problems use different
  // tile lengths).
  const int64_t cref = geo.base + (int64_t)y0 * geo.nx + x0;

  const int tg = tid / (NLINE * NSEG);  // the thread's population in a group (march)
  const int tline = (tid / NSEG) % NLINE;
  // each thread copies, and later reads, only its own staged cells, so its
  // own wait on the copies orders them
  using GR = GroupRec<DIM, QP, QC, G>;
  constexpr int NG = (L::P + G - 1) / G;
  // record component held by each slot of the record buffers (the same in
  // every thread)
  int rcomp[GR::kOn ? GR::NS : 1];
#pragma unroll
  for (int sl = 0; sl < (GR::kOn ? GR::NS : 1); ++sl) rcomp[sl] = -1;
  float refv[G];
  auto prefetch = [&](int gfirst) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int pop = gfirst + g;
      if (pop >= L::P) break;
      const float* __restrict__ srch = Sh + (int64_t)pop * N + geo.base;
      const float* __restrict__ srcl = adv_l + (int64_t)pop * N + geo.base;
#pragma unroll
      for (int j = 0; j < J; ++j)
        if (goff[j] >= 0) {
          cp_async(&sm.rawh[g][tid + j * NT], srch + goff[j]);
          cp_async(&sm.rawl[g][tid + j * NT], srcl + goff[j]);
        }
      refv[g] = DIM == 2 ? Sh[(int64_t)pop * N + cref] : 0.0f;
    }
    if constexpr (GR::kOn) {
#pragma unroll
      for (int sl = 0; sl < GR::NS; ++sl) {
        const int comp = GR::comp(gfirst, sl);
        if (comp < 0 || comp == rcomp[sl]) continue;  // absent, or still there
        rcomp[sl] = comp;
        const float* __restrict__ srch = rbase + (int64_t)comp * N;
        const float* __restrict__ srcl = rbase + (int64_t)(W + comp) * N;
#pragma unroll
        for (int j = 0; j < J; ++j)
          if (goff[j] >= 0) {
            cp_async(&sm.rbh[sl][tid + j * NT], srch + goff[j]);
            cp_async(&sm.rbl[sl][tid + j * NT], srcl + goff[j]);
          }
      }
    }
    cp_async_commit();
  };
  prefetch(group_pop<DIM, QP, QC, G>(0));
  for (int gi = 0; gi < NG; ++gi) {
    const int g0 = group_pop<DIM, QP, QC, G>(gi);  // first population of the group
    // the running explicit parts of the own cells (stage 4, final), early
    float a4v[CPT][G], afv[CPT][G];
    if constexpr (STAGE != kStage3) {
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int pop = g0 + g;
        if (CPT == 2 && pair_vec && pop < L::P) {
          const int64_t e = (int64_t)pop * N + cell[0];
          if (STAGE == kStage4) {
            const float2 v = *reinterpret_cast<const float2*>(p.a4l + e);
            a4v[0][g] = v.x;
            a4v[CPT - 1][g] = v.y;
          }
          const float2 v = *reinterpret_cast<const float2*>(p.afl + e);
          afv[0][g] = v.x;
          afv[CPT - 1][g] = v.y;
          continue;
        }
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
          const bool ok = valid[k] && pop < L::P;
          const int64_t e = (int64_t)pop * N + cell[k];
          a4v[k][g] = (STAGE == kStage4 && ok) ? p.a4l[e] : 0.0f;
          afv[k][g] = ok ? p.afl[e] : 0.0f;
        }
      }
    }
    // ---- stage the group: relaxed advected values - ref on tile + halo
    cp_async_wait_all();
    // With a = sh, b the advected low part and E = Eh + El the equilibrium
    // pair: D = (a - Eh) + (b - El); stage 3 stages F2 - ref = (Eh - ref) +
    // (El + c2 D), stages 4 and final F - ref = (a - ref) + (b - a_ii e_i D).
    // Every operation is rounded on its own, so the paired (packed) and
    // single forms below agree bit for bit.
    auto keep = [&](int g, int j, float w, float d, float a, float b) {
      (&sm.tile[g][0][0])[soff[j]] = w;
      if (oidx[j] >= 0) {
        sm.ownd[g][oidx[j]] = d;
        if constexpr (STAGE == kStage3) sm.ownv[g][oidx[j]] = b;
        if constexpr (STAGE == kFinal) sm.ownv[g][oidx[j]] = a;
      }
    };
    auto relax1 = [&](float a, float b, DF E, float ref, float& d) {
      d = __fadd_rn(__fsub_rn(a, E.hi), __fsub_rn(b, E.lo));
      return STAGE == kStage3 ? __fadd_rn(__fsub_rn(E.hi, ref), fmaf(arelax, d, E.lo))
                              : __fadd_rn(__fsub_rn(a, ref), fmaf(-arelax, d, b));
    };
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int pop = g0 + g;
      if (pop >= L::P) break;
      const float ref = refv[g];
      if constexpr (GR::kOn) {
        const int nphi = DIM == 2 ? QP * QP : QP;
        const bool chi = pop >= nphi;
        const int k = chi ? pop - nphi : pop;
        const int ia = (DIM == 2 ? k % QP : k) - GR::a0(g0);
        // pairs of staged cells; a halo corner or a slot past the staged
        // cells computes on values that are not kept (the last slot's index
        // is clamped into the arrays)
#pragma unroll
        for (int j = 0; j + 1 < J; j += 2) {
          const bool ok0 = goff[j] >= 0, ok1 = goff[j + 1] >= 0;
          const int e0 = tid + j * NT;
          const int e1 = (j + 2) * NT > NSC ? min(tid + (j + 1) * NT, NSC - 1) : tid + (j + 1) * NT;
          const float2 a = make_float2(sm.rawh[g][e0], sm.rawh[g][e1]);
          const float2 b = make_float2(sm.rawl[g][e0], sm.rawl[g][e1]);
          const DF2 A = {make_float2(sm.rbh[ia][e0], sm.rbh[ia][e1]),
                         make_float2(sm.rbl[ia][e0], sm.rbl[ia][e1])};
          DF2 E = A;
          if (DIM == 2 || chi) {
            const DF2 B = {make_float2(sm.rbh[GR::kB][e0], sm.rbh[GR::kB][e1]),
                           make_float2(sm.rbl[GR::kB][e0], sm.rbl[GR::kB][e1])};
            E = pmul2(A, B);
          }
          const float2 d = __fadd2_rn(sub2(a, E.hi), sub2(b, E.lo));
          const float2 w = STAGE == kStage3
                               ? __fadd2_rn(sub2(E.hi, f2s(ref)), __ffma2_rn(f2s(arelax), d, E.lo))
                               : __fadd2_rn(sub2(a, f2s(ref)), __ffma2_rn(f2s(-arelax), d, b));
          if (ok0) keep(g, j, w.x, d.x, a.x, b.x);
          if (ok1) keep(g, j + 1, w.y, d.y, a.y, b.y);
        }
        if constexpr (J % 2 == 1) {
          constexpr int j = J - 1;
          if (goff[j] >= 0) {
            const int e = tid + j * NT;
            const float a = sm.rawh[g][e], b = sm.rawl[g][e];
            DF E = {sm.rbh[ia][e], sm.rbl[ia][e]};
            if (DIM == 2 || chi) E = pmul(E, DF{sm.rbh[GR::kB][e], sm.rbl[GR::kB][e]});
            float d;
            const float w = relax1(a, b, E, ref, d);
            keep(g, j, w, d, a, b);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < J; ++j) {
          if (goff[j] < 0) continue;
          const float a = sm.rawh[g][tid + j * NT], b = sm.rawl[g][tid + j * NT];
          const DF E = eq_from_rec<DIM, QP, QC>(rbase + goff[j], N, pop);
          float d;
          const float w = relax1(a, b, E, ref, d);
          keep(g, j, w, d, a, b);
        }
      }
    }
    __syncthreads();
    if (gi + 1 < NG) prefetch(group_pop<DIM, QP, QC, G>(gi + 1));  // overlaps the march and pass 1
    // ---- every interface value once, marching upwind -> downwind
    {
      const int pop = g0 + tg;
      const bool xline = (DIM == 1) || (tline < TY);
      const float pv = (pop < L::P) ? (xline ? p.pxh[pop] : p.pyh[pop]) : 0.0f;
      const int sgn = (pv >= 0.0f) ? 1 : -1;
      const MarchTask t = march_task(tid, DIM, TX, TY, SEG, SX, sgn);
      if constexpr (DIM == 2) {
        // one segment per line: the flux differences of its cells, the first
        // (in march order) one slot upwind of the first interface's slot
        // when marching downwards
        const int c0 = sgn > 0 ? t.ofirst : t.ofirst - 1;
        float* out = t.xline ? &sm.hx[tg][t.orow][c0] : &sm.hy[tg][t.orow][c0];
        mp9_march_delta_fp32<SEG>(&sm.tile[tg][t.br][t.bc_], t.stride, out, sgn);
      } else {
        mp9_march<SEG>(&sm.tile[tg][t.br][t.bc_], t.stride, &sm.hx[tg][t.orow][t.ofirst], sgn);
      }
    }
    __syncthreads();
    // ---- flux difference and explicit part of the own cells
    if constexpr (CPT == 2) {
      // the thread's two cells in lockstep, as packed binary32 pairs (lane 1
      // of a cell outside the grid computes on unused values, never stored)
      const int o0 = lys[0] * TX + lxs[0], o1 = lys[1] * TX + lxs[1];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int pop = g0 + g;
        if (pop >= L::P) break;
        float2 X;
        const float4 cf = sm.coef[pop];
        const DF cx{cf.x, cf.y};
        if constexpr (DIM == 2) {
          const DF cy{cf.z, cf.w};
          const float2 dx = make_float2(sm.hx[g][lys[0]][lxs[0]], sm.hx[g][lys[1]][lxs[1]]);
          const float2 dy = make_float2(sm.hy[g][lxs[0]][lys[0]], sm.hy[g][lxs[1]][lys[1]]);
          X = __ffma2_rn(f2s(cx.hi), dx, __fmul2_rn(f2s(cx.lo), dx));
          X = __ffma2_rn(f2s(cy.hi), dy, __ffma2_rn(f2s(cy.lo), dy, X));
        } else {
          const float2 dfx = sub2(make_float2(sm.hx[g][lys[0]][lxs[0] + 1], sm.hx[g][lys[1]][lxs[1] + 1]),
                                  make_float2(sm.hx[g][lys[0]][lxs[0]], sm.hx[g][lys[1]][lxs[1]]));
          X = __ffma2_rn(f2s(cx.hi), dfx, __fmul2_rn(f2s(cx.lo), dfx));
        }
        const int64_t e0 = (int64_t)pop * N + cell[0], e1 = (int64_t)pop * N + cell[1];
        // store a pair of the two cells' values: one 8-byte store when the
        // cells are adjacent and aligned, else one per valid cell
        auto put = [&](float* __restrict__ a, float2 v) {
          if (pair_vec) {
            *reinterpret_cast<float2*>(a + e0) = v;
          } else {
            if (valid[0]) a[e0] = v.x;
            if (valid[1]) a[e1] = v.y;
          }
        };
        const float2 d = make_float2(sm.ownd[g][o0], sm.ownd[g][o1]);
        if constexpr (STAGE == kStage3) {
          const float2 l = make_float2(sm.ownv[g][o0], sm.ownv[g][o1]);  // sl
          const float2 r3 = __fadd2_rn(l, __ffma2_rn(f2s(-sc.at32), X, __fmul2_rn(f2s(-sc.k3), d)));
          const float2 a4 = __fadd2_rn(l, __ffma2_rn(f2s(-sc.at42), X, __fmul2_rn(f2s(-sc.k4), d)));
          const float2 af = __fadd2_rn(
              l, __ffma2_rn(f2s(-sc.wt2), X, __ffma2_rn(f2s(-wtl), X, __fmul2_rn(f2s(-sc.kf), d))));
          put(p.r3l, r3);
          put(p.a4l, a4);
          put(p.afl, af);
          accum_low2<DIM, QP, QC>(p, lm2, pop, r3);
        } else if constexpr (STAGE == kStage4) {
          const float2 r4 = __ffma2_rn(f2s(-sc.at43), X,
                                       __ffma2_rn(f2s(-sc.a43e3), d, make_float2(a4v[0][g], a4v[1][g])));
          const float2 af = __ffma2_rn(
              f2s(-sc.wt3), X,
              __ffma2_rn(f2s(-wtl), X,
                         __ffma2_rn(f2s(-sc.w3e3), d, make_float2(afv[0][g], afv[1][g]))));
          put(p.a4l, r4);
          put(p.afl, af);
          accum_low2<DIM, QP, QC>(p, lm2, pop, r4);
        } else {
          // F^{n+1} = sh + t with t = afl - w4 e4 D4 - wt4 X4, renormalised by
          // TwoSum into the next buffer
          const float2 t = __ffma2_rn(
              f2s(-sc.wt4), X,
              __ffma2_rn(f2s(-wtl), X,
                         __ffma2_rn(f2s(-sc.w4e4), d, make_float2(afv[0][g], afv[1][g]))));
          const float2 a = make_float2(sm.ownv[g][o0], sm.ownv[g][o1]);  // sh
          const float2 s = __fadd2_rn(a, t);
          const float2 bb = sub2(s, a);
          const float2 er = __fadd2_rn(sub2(a, sub2(s, bb)), sub2(t, bb));
          put(p.nh, s);
          put(p.nl, er);
          accumulate2<DIM, QP, QC>(p, mom2, pop, s);
          accum_low2<DIM, QP, QC>(p, lm2, pop, er);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        if (!valid[k]) continue;
        const int lx = lxs[k], ly = lys[k], o = ly * TX + lx;
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int pop = g0 + g;
          if (pop >= L::P) break;
          float X;
          const float4 cf = sm.coef[pop];
          const DF cx{cf.x, cf.y};
          if constexpr (DIM == 2) {
            const DF cy{cf.z, cf.w};
            const float dx = sm.hx[g][ly][lx], dy = sm.hy[g][lx][ly];
            X = fmaf(cx.hi, dx, __fmul_rn(cx.lo, dx));
            X = fmaf(cy.hi, dy, fmaf(cy.lo, dy, X));
          } else {
            const float dfx = __fsub_rn(sm.hx[g][ly][lx + 1], sm.hx[g][ly][lx]);
            X = fmaf(cx.hi, dfx, __fmul_rn(cx.lo, dfx));
          }
          const int64_t e = (int64_t)pop * N + cell[k];
          const float d = sm.ownd[g][o];
          if constexpr (STAGE == kStage3) {
            const float l = sm.ownv[g][o];
            const float r3 = __fadd_rn(l, fmaf(-sc.at32, X, __fmul_rn(-sc.k3, d)));
            p.r3l[e] = r3;
            p.a4l[e] = __fadd_rn(l, fmaf(-sc.at42, X, __fmul_rn(-sc.k4, d)));
            p.afl[e] = __fadd_rn(l, fmaf(-sc.wt2, X, fmaf(-wtl, X, __fmul_rn(-sc.kf, d))));
            accum_low<DIM, QP, QC>(p, lm[k], pop, r3);
          } else if constexpr (STAGE == kStage4) {
            const float r4 = fmaf(-sc.at43, X, fmaf(-sc.a43e3, d, a4v[k][g]));
            p.a4l[e] = r4;
            p.afl[e] = fmaf(-sc.wt3, X, fmaf(-wtl, X, fmaf(-sc.w3e3, d, afv[k][g])));
            accum_low<DIM, QP, QC>(p, lm[k], pop, r4);
          } else {
            const float t = fmaf(-sc.wt4, X, fmaf(-wtl, X, fmaf(-sc.w4e4, d, afv[k][g])));
            const float a = sm.ownv[g][o];
            const float s = __fadd_rn(a, t);
            const float bb = __fsub_rn(s, a);
            const float er = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(t, bb));
            p.nh[e] = s;
            p.nl[e] = er;
            accumulate<DIM, QP, QC>(p, mom[k], pop, s);
            accum_low<DIM, QP, QC>(p, lm[k], pop, er);
          }
        }
      }
    }
    __syncthreads();
  }
  if constexpr (CPT == 2) {
    lm[0] = MomL{lm2.n.x, lm2.jx.x, lm2.jy.x, lm2.e.x};
    lm[1] = MomL{lm2.n.y, lm2.jx.y, lm2.jy.y, lm2.e.y};
    mom[0] = lane(mom2, 0);
    mom[1] = lane(mom2, 1);
  }
  // ---- per cell: binary64 moments of the stage's explicit part (or of the
  // new state) and the record of its equilibrium (the next kernel relaxes)
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    if (!valid[k]) continue;
    const int64_t c = cell[k];
    double mh[4];
    if constexpr (STAGE == kFinal) {
      const Moments m = to_fp64(mom[k]);
      mh[0] = m.n;
      mh[1] = m.jx;
      mh[2] = m.jy;
      mh[3] = m.e;
#pragma unroll
      for (int i = 0; i < 4; ++i) p.mhi[i * N + c] = mh[i];
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) mh[i] = p.mhi[i * N + c];
    }
    finish_cell<DIM, QP, QC>(p, geo.kchi, geo.invDK, geo.prob, mh[0] + (double)lm[k].n,
                             mh[1] + (double)lm[k].jx, mh[2] + (double)lm[k].jy,
                             mh[3] + (double)lm[k].e, rout, c);
  }
}

template <int DIM, int QP, int QC, int STAGE, int VAR = 0>
__global__ void __launch_bounds__(TileCfg<DIM, VAR>::NT,
                                  DIM == 2 ? 3 : (TileCfg<DIM, VAR>::NT >= 128 ? 4 : 8))
    mixed_stage_kernel(const __grid_constant__ DevParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  auto& sm = *reinterpret_cast<MixSmem<DIM, QP, QC, VAR, STAGE>*>(smraw);
  const Geo geo{p.nx, p.ny, 0, p.kchi, p.invDK, p.dtdx, p.dtdy, -1};
  mixed_tile<DIM, QP, QC, STAGE, VAR>(p, geo, blockIdx.x * TileCfg<DIM, VAR>::TX,
                                      blockIdx.y * TileCfg<DIM, VAR>::TY, sm);
}

template <int QP, int QC, int STAGE, int VAR>
__global__ void __launch_bounds__(TileCfg<1, VAR>::NT, 4)
    mixed_batch_kernel(const __grid_constant__ DevParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  auto& sm = *reinterpret_cast<MixSmem<1, QP, QC, VAR, STAGE>*>(smraw);
  for (int w = blockIdx.x; w < p.nwork; w += gridDim.x) {
    const WorkItem it = p.work[w];
    const BatchProblem& bp = p.probs[it.prob];
    const Geo geo{bp.nx, 1, bp.base, bp.kchi, bp.invDK, bp.dtdx, 0.0, it.prob};
    mixed_tile<1, QP, QC, STAGE, VAR>(p, geo, it.x0, 0, sm);
  }
}

// problem of cell c (problems sorted by base)
__device__ __forceinline__ int problem_of(const DevParams& p, int64_t c) {
  int lo = 0, hi = p.nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (p.probs[mid].base <= c) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// After fdlb_init_riemann or fdlb_set_state: mhi and the record of F^n, with
// the final stage's sums in the final stage's population order (so that a
// state set from a copy continues bit for bit).  G is the group size of the
// kernels the context runs.
template <int DIM, int QP, int QC, int G>
__global__ void mixed_prep_kernel(const __grid_constant__ DevParams p) {
  using L = Lat<DIM, QP, QC>;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  MomentsF m = {};
  MomL lm = {};
  constexpr int NG = (L::P + G - 1) / G;
  for (int gi = 0; gi < NG; ++gi) {
    const int g0 = group_pop<DIM, QP, QC, G>(gi);
    for (int g = 0; g < G && g0 + g < L::P; ++g) {
      const int pop = g0 + g;
      accumulate<DIM, QP, QC>(p, m, pop, p.sh[pop * p.N + c]);
      accum_low<DIM, QP, QC>(p, lm, pop, p.sl[pop * p.N + c]);
    }
  }
  Geo geo{p.nx, p.ny, 0, p.kchi, p.invDK, p.dtdx, p.dtdy, -1};
  if (p.nprob > 0) {
    const int b = problem_of(p, c);
    geo.kchi = p.probs[b].kchi;
    geo.invDK = p.probs[b].invDK;
    geo.prob = b;
  }
  const Moments mh = to_fp64(m);
  p.mhi[c] = mh.n;
  p.mhi[p.N + c] = mh.jx;
  p.mhi[2 * p.N + c] = mh.jy;
  p.mhi[3 * p.N + c] = mh.e;
  finish_cell<DIM, QP, QC>(p, geo.kchi, geo.invDK, geo.prob, mh.n + (double)lm.n,
                           mh.jx + (double)lm.jx, mh.jy + (double)lm.jy, mh.e + (double)lm.e,
                           p.erec[0], c);
}

template <int DIM, int QP, int QC, int VAR, int STAGE>
constexpr int smem_bytes() {
  return (int)sizeof(MixSmem<DIM, QP, QC, VAR, STAGE>);
}

template <int DIM, int QP, int QC, int VAR>
int setup_tv() {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mixed_stage_kernel<DIM, QP, QC, kStage3, VAR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<DIM, QP, QC, VAR, kStage3>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mixed_stage_kernel<DIM, QP, QC, kStage4, VAR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<DIM, QP, QC, VAR, kStage4>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mixed_stage_kernel<DIM, QP, QC, kFinal, VAR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<DIM, QP, QC, VAR, kFinal>());
  return (int)e;
}

template <int DIM, int QP, int QC>
int setup_t() {
  int e = setup_tv<DIM, QP, QC, 0>();
  if constexpr (DIM == 1) {
    if (!e) e = setup_tv<1, QP, QC, 1>();
    if (!e) e = setup_tv<1, QP, QC, 3>();
    if (!e) e = setup_tv<1, QP, QC, 4>();
  }
  return e;
}

template <int QP, int QC, int VAR>
int setup_batch_v() {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mixed_batch_kernel<QP, QC, kStage3, VAR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<1, QP, QC, VAR, kStage3>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mixed_batch_kernel<QP, QC, kStage4, VAR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<1, QP, QC, VAR, kStage4>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mixed_batch_kernel<QP, QC, kFinal, VAR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<1, QP, QC, VAR, kFinal>());
  return (int)e;
}

template <int DIM, int QP, int QC, int VAR>
int launch_tv(const DevParams& p, int stage, cudaStream_t s) {
  using C = TileCfg<DIM, VAR>;
  const dim3 grid((p.nx + C::TX - 1) / C::TX, DIM == 2 ? (p.ny + C::TY - 1) / C::TY : 1);
  switch (stage) {
    case kStage3:
      mixed_stage_kernel<DIM, QP, QC, kStage3, VAR>
          <<<grid, C::NT, smem_bytes<DIM, QP, QC, VAR, kStage3>(), s>>>(p);
      break;
    case kStage4:
      mixed_stage_kernel<DIM, QP, QC, kStage4, VAR>
          <<<grid, C::NT, smem_bytes<DIM, QP, QC, VAR, kStage4>(), s>>>(p);
      break;
    default:
      mixed_stage_kernel<DIM, QP, QC, kFinal, VAR>
          <<<grid, C::NT, smem_bytes<DIM, QP, QC, VAR, kFinal>(), s>>>(p);
      break;
  }
  return (int)cudaGetLastError();
}

template <int DIM, int QP, int QC, int G>
int launch_prep(const DevParams& p, cudaStream_t s) {
  const int nt = 128;
  const int64_t nb = (p.N + nt - 1) / nt;
  mixed_prep_kernel<DIM, QP, QC, G><<<(unsigned)nb, nt, 0, s>>>(p);
  return (int)cudaGetLastError();
}

template <int DIM, int QP, int QC>
int launch_t(const DevParams& p, int stage, cudaStream_t s) {
  if constexpr (DIM == 1) {
    // 1-D problems pick their tile shape by length (single_1d_variant)
    switch (single_1d_variant(p.nx)) {
      case 1:
        return stage == kPrep ? launch_prep<1, QP, QC, TileCfg<1, 1>::G>(p, s)
                              : launch_tv<1, QP, QC, 1>(p, stage, s);
      case 3:
        return stage == kPrep ? launch_prep<1, QP, QC, TileCfg<1, 3>::G>(p, s)
                              : launch_tv<1, QP, QC, 3>(p, stage, s);
      case 4:
        return stage == kPrep ? launch_prep<1, QP, QC, TileCfg<1, 4>::G>(p, s)
                              : launch_tv<1, QP, QC, 4>(p, stage, s);
      default:
        return stage == kPrep ? launch_prep<1, QP, QC, TileCfg<1, 0>::G>(p, s)
                              : launch_tv<1, QP, QC, 0>(p, stage, s);
    }
  }
  if (stage == kPrep) return launch_prep<DIM, QP, QC, TileCfg<DIM, 0>::G>(p, s);
  return launch_tv<DIM, QP, QC, 0>(p, stage, s);
}

template <int QP, int QC, int VAR>
int launch_batch_v(const DevParams& p, int stage, cudaStream_t s) {
  using C = TileCfg<1, VAR>;
  const int grid = p.bgrid > 0 ? p.bgrid : 1;
  switch (stage) {
    case kPrep:
      return launch_prep<1, QP, QC, C::G>(p, s);
    case kStage3:
      mixed_batch_kernel<QP, QC, kStage3, VAR>
          <<<grid, C::NT, smem_bytes<1, QP, QC, VAR, kStage3>(), s>>>(p);
      break;
    case kStage4:
      mixed_batch_kernel<QP, QC, kStage4, VAR>
          <<<grid, C::NT, smem_bytes<1, QP, QC, VAR, kStage4>(), s>>>(p);
      break;
    default:
      mixed_batch_kernel<QP, QC, kFinal, VAR>
          <<<grid, C::NT, smem_bytes<1, QP, QC, VAR, kFinal>(), s>>>(p);
      break;
  }
  return (int)cudaGetLastError();
}

template <int QP, int QC>
int launch_batch_t(const DevParams& p, int stage, cudaStream_t s) {
  switch (p.variant) {
    case 1: return launch_batch_v<QP, QC, 1>(p, stage, s);
    case 2: return launch_batch_v<QP, QC, 2>(p, stage, s);
    default: return launch_batch_v<QP, QC, 0>(p, stage, s);
  }
}

// ---- the state as binary64 values (fdlb_get_state / fdlb_set_state) ------

__global__ void pair_to_double_kernel(const float* __restrict__ hi, const float* __restrict__ lo,
                                      double* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)hi[i] + (double)lo[i];  // exact: |lo| <= ulp(hi)/2
}

__global__ void double_to_pair_kernel(const double* __restrict__ in, float* __restrict__ hi,
                                      float* __restrict__ lo, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = in[i];
    const float h = (float)v;
    hi[i] = h;
    lo[i] = (float)(v - (double)h);
  }
}

}  // namespace

int mixed_record_width(int d, int Qp, int Qc) {
#define X(D_, P_, C_) \
  if (d == D_ && Qp == P_ && Qc == C_) return RecLayout<D_, P_, C_>::W;
  FDLB_LATTICES(X)
#undef X
  return 0;
}

int mixed_setup(const DevParams& p) {
  if (p.nprob > 0) {
#define X(P_, C_)                                                                   \
  if (p.Qp == P_ && p.Qc == C_) {                                                   \
    int e = setup_batch_v<P_, C_, 0>();                                             \
    if (!e) e = setup_batch_v<P_, C_, 1>();                                         \
    if (!e) e = setup_batch_v<P_, C_, 2>();                                         \
    return e;                                                                       \
  }
    FDLB_BATCH_LATTICES(X)
#undef X
    return (int)cudaErrorInvalidValue;
  }
#define X(D_, P_, C_) \
  if (p.d == D_ && p.Qp == P_ && p.Qc == C_) return setup_t<D_, P_, C_>();
  FDLB_LATTICES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int launch_mixed_stage(const DevParams& p, int stage, cudaStream_t s) {
#define X(D_, P_, C_) \
  if (p.d == D_ && p.Qp == P_ && p.Qc == C_) return launch_t<D_, P_, C_>(p, stage, s);
  FDLB_LATTICES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int launch_mixed_batch_stage(const DevParams& p, int stage, cudaStream_t s) {
#define X(P_, C_) \
  if (p.Qp == P_ && p.Qc == C_) return launch_batch_t<P_, C_>(p, stage, s);
  FDLB_BATCH_LATTICES(X)
#undef X
  return (int)cudaErrorInvalidValue;
}

int launch_pair_to_double(const float* hi, const float* lo, double* out, int64_t n,
                          cudaStream_t s) {
  pair_to_double_kernel<<<1024, 256, 0, s>>>(hi, lo, out, n);
  return (int)cudaGetLastError();
}

int launch_double_to_pair(const double* in, float* hi, float* lo, int64_t n, cudaStream_t s) {
  double_to_pair_kernel<<<1024, 256, 0, s>>>(in, hi, lo, n);
  return (int)cudaGetLastError();
}

}  // namespace fdlb
