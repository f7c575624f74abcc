// fdlb_mixed.cu -- binary32 stage kernels of the IMEX step (FDLB_MIXED):
// one pass over memory per advected stage.
//
// The binary64 kernels (fdlb_kernels.cu) relax a stage in a second pass over
// values parked in the output arrays, because the equilibrium of a cell needs
// the moments of all its populations.  Here the relaxation of stage i is
// applied by the kernel of stage i+1, when it loads the advected array:
//   * every kernel writes the unrelaxed explicit part R_i of its stage, sums
//     the moments of R_i per cell (Eq. Moments_discrete, compensated binary32
//     pairs), and stores a record of the cell's equilibrium factors
//     (Eq. gExpanded, in binary32-pair arithmetic of about 48 significant
//     bits, each factor rounded once to binary32);
//   * the next kernel forms the relaxed values from R_i and the record as it
//     stages the tile and its halo (Sec. III closed forms):
//       stage 3 stages F2 = E0 + c2 (F^n - E0) from F^n,
//       stage 4 stages F3 = R3 - a33 e3 (R3 - E3) from R3,
//       the final stage stages F4 = R4 - a44 e4 (R4 - E4) from R4,
//     and uses D = F^n - E0, D3 = R3 - E3, D4 = R4 - E4 at its own cells.
// Arrays read and written per population and step: stage 3 reads F^n and
// writes R3, A4', Af'; stage 4 reads R3, A4', Af' and writes R4, Af''; the
// final stage reads R4, Af'' and writes F^{n+1} -- 6 reads and 6 writes of
// 4 bytes, plus one record per cell and kernel.
#include "fdlb_device.cuh"

namespace fdlb {
namespace {

// Components of a cell's record.  phi^eq(kx, ky) = A[kx] * B[ky] with
// A = n g_x, B = g_y (1-D: A[k]); chi^eq(qx, qy) = C * A[qx] * B[qy] with
// C = (D+K-d) T when Qchi = Qphi, else Hx[qx] * Hy[qy] with Hx = nchi h_x.
// 2-D records with Qchi = Qphi also hold CB[ky] = C B[ky] (each rounded once),
// so that chi^eq = A[qx] * CB[qy] takes the same two factors as phi^eq.
template <int DIM, int QP, int QC>
struct RecLayout {
  static constexpr bool kSame = QP == QC;
  static constexpr int kChi = DIM == 1 ? QP : 2 * QP;  // first chi component
  static constexpr bool kCB = DIM == 2 && kSame;
  static constexpr int kCBo = kChi + 1;               // first CB component
  static constexpr int W = kSame ? kChi + 1 + (kCB ? QP : 0) : kChi + (DIM == 1 ? QC : 2 * QC);
  static_assert(!kCB || kCBo + QP == W, "CB components close the record");
};

// Equilibrium of population pop from a record whose components lie `stride`
// floats apart (read through the read-only data cache).
template <int DIM, int QP, int QC>
__device__ __forceinline__ float eq_from_rec(const float* __restrict__ rec, int64_t stride,
                                             int pop) {
  using R = RecLayout<DIM, QP, QC>;
  using L = Lat<DIM, QP, QC>;
  if (pop < L::NPHI) {
    if constexpr (DIM == 1) return rec[pop * stride];
    else return rec[(pop % QP) * stride] * rec[(QP + pop / QP) * stride];
  }
  const int q = pop - L::NPHI;
  if constexpr (R::kSame) {
    if constexpr (DIM == 1) return rec[R::kChi * stride] * rec[q * stride];
    else return rec[R::kChi * stride] * (rec[(q % QP) * stride] * rec[(QP + q / QP) * stride]);
  } else {
    if constexpr (DIM == 1) return rec[(R::kChi + q) * stride];
    else return rec[(R::kChi + q % QC) * stride] * rec[(R::kChi + QC + q / QC) * stride];
  }
}

// ---- binary32 pairs: x = hi + lo with about 48 significant bits ----------
// The records' Hermite factors are evaluated in this arithmetic on the
// binary32 pipe.  GB300's binary64 pipe runs at 1/64 of the binary32 rate;
// evaluated in binary64, the factors of a 1-D cell (16 populations) would
// cost more pipe time than all of the cell's population work.  The pair
// arithmetic is the classical error-free one (Dekker, Knuth): TwoSum for
// additions, the fused multiply-add for the exact product error; the
// intrinsics keep the compiler from contracting the error terms away.
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
__device__ __forceinline__ float df_round(DF x) { return __fadd_rn(x.hi, x.lo); }

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
// apart), in pair arithmetic, each component rounded once to binary32.
template <int DIM, int QP, int QC>
__device__ __forceinline__ void write_record(const DevParams& p, DF kchi, DF n, DF ux, DF uy, DF T,
                                             float* __restrict__ rec, int64_t cell, int64_t N) {
  using R = RecLayout<DIM, QP, QC>;
  const DF one{1.0f, 0.0f};
  DF g[QP];
  axis_g_df<QP>(p.wHph, p.wHpl, ux, T, n, g);
#pragma unroll
  for (int k = 0; k < QP; ++k) rec[k * N + cell] = df_round(g[k]);
  if constexpr (DIM == 2) {
    axis_g_df<QP>(p.wHph, p.wHpl, uy, T, one, g);
#pragma unroll
    for (int k = 0; k < QP; ++k) rec[(QP + k) * N + cell] = df_round(g[k]);
  }
  const DF kT = df_mul(kchi, T);
  if constexpr (R::kSame) {
    rec[R::kChi * N + cell] = df_round(kT);
    if constexpr (R::kCB) {  // g holds the y factors B
#pragma unroll
      for (int k = 0; k < QP; ++k) rec[(R::kCBo + k) * N + cell] = df_round(df_mul(kT, g[k]));
    }
  } else {
    DF h[QC];
    axis_g_df<QC>(p.wHch, p.wHcl, ux, T, df_mul(kT, n), h);
#pragma unroll
    for (int q = 0; q < QC; ++q) rec[(R::kChi + q) * N + cell] = df_round(h[q]);
    if constexpr (DIM == 2) {
      axis_g_df<QC>(p.wHch, p.wHcl, uy, T, one, h);
#pragma unroll
      for (int q = 0; q < QC; ++q) rec[(R::kChi + QC + q) * N + cell] = df_round(h[q]);
    }
  }
}

// Moments of a cell -> validity flags and record: n, u = j/n and
// T = (E - j u)/((D+K) n) (Eq. Moments_discrete and the temperature
// definition) from the compensated sums, in pair arithmetic.  The reciprocal
// is one Newton step from the binary32 one.
template <int DIM, int QP, int QC>
__device__ __forceinline__ void finish_cell(const DevParams& p, DF kchi, DF invDK, int prob,
                                            const MomentsF& m, float* __restrict__ rec,
                                            int64_t cell) {
  const DF zero{0.0f, 0.0f};
  const DF n = df_add(DF{m.nh, 0.0f}, DF{m.nl, 0.0f});
  const DF jx = df_add(DF{m.jxh, 0.0f}, DF{m.jxl, 0.0f});
  const DF jy = DIM == 2 ? df_add(DF{m.jyh, 0.0f}, DF{m.jyl, 0.0f}) : zero;
  const DF e = df_add(DF{m.eh, 0.0f}, DF{m.el, 0.0f});
  const float r0 = __frcp_rn(n.hi);
  const DF inv_n = df_add(DF{r0, 0.0f},
                          df_mul(DF{r0, 0.0f}, df_add(DF{1.0f, 0.0f}, df_neg(df_mul(n, DF{r0, 0.0f})))));
  const DF ux = df_mul(jx, inv_n);
  const DF uy = DIM == 2 ? df_mul(jy, inv_n) : zero;
  DF ke = df_add(e, df_neg(df_mul(jx, ux)));
  if constexpr (DIM == 2) ke = df_add(ke, df_neg(df_mul(jy, uy)));
  const DF T = df_mul(df_mul(ke, inv_n), invDK);
  const bool ok = n.hi > 0.0f && T.hi > 0.0f && isfinite(n.hi) && isfinite(T.hi) &&
                  isfinite(ux.hi) && isfinite(uy.hi);
  if (!ok) {
    atomicOr(p.status, 1u);
    if (prob >= 0) atomicOr(&p.pstatus[prob], 1u);
  }
  write_record<DIM, QP, QC>(p, kchi, n, ux, uy, T, rec, cell, p.N);
}

// Record prefetch plan of a population group, for lattices with Qchi = Qphi
// whose groups align with rows of the velocity grid ((8, 8) with groups of 4
// in 2-D; groups of 8 or 16 in 1-D).  Slot s of the group's buffer holds one
// record component: slots 0..NA-1 the x factors A of the group's columns,
// then slot kB the second factor: in 2-D B of the group's row (phi) or CB
// (chi), in 1-D the chi factor C.
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

template <int DIM, int QP, int QC, int VAR, int STAGE>
struct MixSmem {
  using C = TileCfg<DIM, VAR>;
  static constexpr int SXH = C::TX + 2 * H;             // staged columns
  static constexpr int SX = SXH + (DIM == 2 ? 1 : 0);   // tile row pitch
  static constexpr int SY = DIM == 2 ? C::TY + 2 * H : 1;
  // staged cells: tile + halo without the 2-D corner blocks, which feed no
  // line (rows 0..H-1 and H+TY.. take the tile's columns only)
  static constexpr int NSC = DIM == 2 ? C::TY * SXH + 2 * H * C::TX : SXH;
  float raw[C::G][NSC];                // the group's advected values as loaded
  // the group's record components (GroupRec plan), as loaded
  float rbuf[GroupRec<DIM, QP, QC, C::G>::kOn ? GroupRec<DIM, QP, QC, C::G>::NS : 1]
            [GroupRec<DIM, QP, QC, C::G>::kOn ? NSC : 1];
  float tile[C::G][SY][SX];            // relaxed advected populations
  float hx[C::G][C::TY][C::TX + 1];    // interface values along x
  float hy[DIM == 2 ? C::G : 1][DIM == 2 ? C::TX : 1][C::TY + 1];
  float ownd[C::G][C::TY * C::TX];     // R - F_eq of the own cells
  // stage 3 only: F^n of the own cells
  float ownv[STAGE == kStage3 ? C::G : 1][STAGE == kStage3 ? C::TY * C::TX : 1];
};

// One tile of one stage.  Ends with every thread past its last use of the
// shared memory, so a persistent CTA may start its next tile at once.
template <int DIM, int QP, int QC, int STAGE, int VAR>
__device__ __forceinline__ void mixed_tile(const DevParams& p, const Geo& geo, int x0, int y0,
                                           MixSmem<DIM, QP, QC, VAR, STAGE>& sm) {
  using C = TileCfg<DIM, VAR>;
  using L = Lat<DIM, QP, QC>;
  using M = MixSmem<DIM, QP, QC, VAR, STAGE>;
  constexpr int TX = C::TX, TY = C::TY, NT = C::NT, G = C::G, SEG = C::SEG;
  constexpr int SX = M::SX, SXH = M::SXH, NSC = M::NSC;
  constexpr int CELLS = TX * TY;
  constexpr int CPT = (CELLS + NT - 1) / NT;
  constexpr int NSEG = (TX + 1) / SEG;
  static_assert(NSEG * SEG == TX + 1, "segments tile the line");
  constexpr int NLINE = DIM == 2 ? TX + TY : 1;
  static_assert(G * NLINE * NSEG == NT, "one march task per thread");
  constexpr int J = (NSC + NT - 1) / NT;  // staged cells per thread

  float* __restrict__ const F = (float*)p.F;
  float* __restrict__ const R3 = (float*)p.F3;
  float* __restrict__ const A4 = (float*)p.A4;
  float* __restrict__ const Af = (float*)p.Af;
  const float* __restrict__ const rin =
      p.erec[STAGE == kStage3 ? 0 : (STAGE == kStage4 ? 1 : 2)];
  float* __restrict__ const rout = p.erec[STAGE == kStage3 ? 1 : (STAGE == kStage4 ? 2 : 0)];
  const float* __restrict__ const adv = STAGE == kStage3 ? F : (STAGE == kStage4 ? R3 : A4);
  const int tid = threadIdx.x;
  const int64_t N = p.N;

  // this thread's staged cells: tile offset, cell offset from geo.base
  // (-1: none), own-cell index (-1: halo)
  int soff[J], goff[J], oidx[J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int e = tid + j * NT;
    // staged cell e (NSC of them): 2-D in three blocks -- rows above the tile
    // (tile columns only), the tile's rows with both side halos, rows below
    int r, c;
    if (DIM == 1) {
      r = 0;
      c = e;
    } else if (e < H * TX) {
      r = e / TX;
      c = H + e % TX;
    } else if (e < H * TX + TY * SXH) {
      r = H + (e - H * TX) / SXH;
      c = (e - H * TX) % SXH;
    } else {
      r = H + TY + (e - H * TX - TY * SXH) / TX;
      c = H + (e - H * TX - TY * SXH) % TX;
    }
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
    const int c = tid + k * NT;
    lxs[k] = c % TX;
    lys[k] = c / TX;
    valid[k] = (c < CELLS) && (x0 + lxs[k] < geo.nx) && (y0 + lys[k] < geo.ny);
    cell[k] = geo.base + (int64_t)(y0 + lys[k]) * geo.nx + (x0 + lxs[k]);
  }
  MomentsF mom[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) mom[k] = {};
  MomentsF2 mom2 = {};  // the two cells' sums when CPT == 2
  const CoefS<float> sc(p.sc);
  const float arelax = STAGE == kStage3 ? sc.c2 : (STAGE == kStage4 ? sc.a33e3 : sc.a44e4);
  const float dtdx = (float)geo.dtdx, dtdy = (float)geo.dtdy;
  const DF kchi_df = df_of(geo.kchi), invDK_df = df_of(geo.invDK);
  const float* __restrict__ const rbase = rin + geo.base;

  const int tg = tid / (NLINE * NSEG);
  const int tline = (tid / NSEG) % NLINE;
  const int tseg = tid % NSEG;
  // each thread copies, and later reads, only its own staged cells, so its
  // own wait on the copies orders them
  using GR = GroupRec<DIM, QP, QC, G>;
  // Group order.  2-D groups with a record plan run x-block-major: the 8
  // groups that share the x factors A of one block of G columns come one
  // after another (rows ky = 0..QP-1), phi before chi, so that only B (and C
  // once) change from one group to the next.  Otherwise groups run in
  // population order.
  constexpr int NG = (L::P + G - 1) / G;
  auto gpop = [](int gi) -> int {
    if constexpr (DIM == 2 && GR::kOn) {
      constexpr int per_half = L::NPHI / G;
      const int half = gi / per_half, r = gi % per_half;
      return half * L::NPHI + (r % QP) * QP + (r / QP) * G;
    } else {
      return gi * G;
    }
  };
  // record component held by each slot of sm.rbuf (the same in every thread)
  int rcomp[GR::kOn ? GR::NS : 1];
#pragma unroll
  for (int sl = 0; sl < (GR::kOn ? GR::NS : 1); ++sl) rcomp[sl] = -1;
  auto prefetch = [&](int gfirst) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int pop = gfirst + g;
      if (pop >= L::P) break;
      const float* __restrict__ src = adv + (int64_t)pop * N + geo.base;
#pragma unroll
      for (int j = 0; j < J; ++j)
        if (goff[j] >= 0) cp_async(&sm.raw[g][tid + j * NT], src + goff[j]);
    }
    if constexpr (GR::kOn) {
#pragma unroll
      for (int sl = 0; sl < GR::NS; ++sl) {
        const int comp = GR::comp(gfirst, sl);
        if (comp < 0 || comp == rcomp[sl]) continue;  // absent, or still there
        rcomp[sl] = comp;
        const float* __restrict__ src = rbase + (int64_t)comp * N;
#pragma unroll
        for (int j = 0; j < J; ++j)
          if (goff[j] >= 0) cp_async(&sm.rbuf[sl][tid + j * NT], src + goff[j]);
      }
    }
    cp_async_commit();
  };
  prefetch(gpop(0));
  for (int gi = 0; gi < NG; ++gi) {
    const int g0 = gpop(gi);  // first population of the group
    // the running explicit parts of the own cells (stage 4, final), early
    float a4v[CPT][G], afv[CPT][G];
    if constexpr (STAGE != kStage3) {
#pragma unroll
      for (int k = 0; k < CPT; ++k)
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int pop = g0 + g;
          const bool ok = valid[k] && pop < L::P;
          const int64_t e = (int64_t)pop * N + cell[k];
          a4v[k][g] = (STAGE == kStage4 && ok) ? A4[e] : 0.0f;
          afv[k][g] = ok ? Af[e] : 0.0f;
        }
    }
    // ---- stage the group: relaxed advected values on tile + halo
    cp_async_wait_all();
    // The equilibrium is A B (phi) or A CB (chi) from the record slots in
    // 2-D, A (phi) or C A (chi) in 1-D,
    // D = R - F_eq, and stage 3 stages F2 = E0 + c2 D, stages 4 and final
    // F = R - a_ii e_i D; every operation is rounded on its own, so the
    // paired (packed) and single forms below agree bit for bit.
    auto keep = [&](int g, int j, float w, float d, float v) {
      (&sm.tile[g][0][0])[soff[j]] = w;
      if (oidx[j] >= 0) {
        sm.ownd[g][oidx[j]] = d;
        if constexpr (STAGE == kStage3) sm.ownv[g][oidx[j]] = v;
      }
    };
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int pop = g0 + g;
      if (pop >= L::P) break;
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
          const float2 v = make_float2(sm.raw[g][e0], sm.raw[g][e1]);
          float2 fe = make_float2(sm.rbuf[ia][e0], sm.rbuf[ia][e1]);
          if constexpr (DIM == 2)
            fe = __fmul2_rn(fe, make_float2(sm.rbuf[GR::kB][e0], sm.rbuf[GR::kB][e1]));
          else if (chi)
            fe = __fmul2_rn(make_float2(sm.rbuf[GR::kB][e0], sm.rbuf[GR::kB][e1]), fe);
          const float2 d = sub2(v, fe);
          const float2 w = STAGE == kStage3 ? __ffma2_rn(f2s(arelax), d, fe)
                                            : __ffma2_rn(f2s(-arelax), d, v);
          if (ok0) keep(g, j, w.x, d.x, v.x);
          if (ok1) keep(g, j + 1, w.y, d.y, v.y);
        }
        if constexpr (J % 2 == 1) {
          constexpr int j = J - 1;
          if (goff[j] >= 0) {
            const int e = tid + j * NT;
            const float v = sm.raw[g][e];
            float fe = sm.rbuf[ia][e];
            if constexpr (DIM == 2) fe = __fmul_rn(fe, sm.rbuf[GR::kB][e]);
            else if (chi) fe = __fmul_rn(sm.rbuf[GR::kB][e], fe);
            const float d = __fsub_rn(v, fe);
            keep(g, j, STAGE == kStage3 ? fmaf(arelax, d, fe) : fmaf(-arelax, d, v), d, v);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < J; ++j) {
          if (goff[j] < 0) continue;
          const float v = sm.raw[g][tid + j * NT];
          const float fe = eq_from_rec<DIM, QP, QC>(rbase + goff[j], N, pop);
          const float d = __fsub_rn(v, fe);
          keep(g, j, STAGE == kStage3 ? fmaf(arelax, d, fe) : fmaf(-arelax, d, v), d, v);
        }
      }
    }
    __syncthreads();
    if (gi + 1 < NG) prefetch(gpop(gi + 1));  // overlaps the march and pass 1
    // ---- every interface value once, marching upwind -> downwind
    {
      const int pop = g0 + tg;
      const bool xline = (DIM == 1) || (tline < TY);
      const float pv = (pop < L::P) ? (xline ? p.pxh[pop] : p.pyh[pop]) : 0.0f;
      const int sgn = (pv >= 0.0f) ? 1 : -1;
      const int i0 = tseg * SEG;
      const int first = (sgn > 0) ? i0 : i0 + SEG - 1;
      const int up = ((sgn > 0) ? first - 1 : first) + H;
      const int r = (DIM == 2 && xline) ? tline : 0;
      const int c = xline ? 0 : tline - TY;
      const float* base = xline ? &sm.tile[tg][r + (DIM == 2 ? H : 0)][up] : &sm.tile[tg][up][c + H];
      const int stride = xline ? 1 : SX;
      float* out = xline ? &sm.hx[tg][r][first] : &sm.hy[tg][c][first];
      mp9_march<SEG>(base, sgn * stride, out, sgn);
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
        const float2 dfx = sub2(make_float2(sm.hx[g][lys[0]][lxs[0] + 1], sm.hx[g][lys[1]][lxs[1] + 1]),
                                make_float2(sm.hx[g][lys[0]][lxs[0]], sm.hx[g][lys[1]][lxs[1]]));
        float2 X = __fmul2_rn(f2s(dtdx * p.pxh[pop]), dfx);
        if constexpr (DIM == 2) {
          const float2 dfy = sub2(make_float2(sm.hy[g][lxs[0]][lys[0] + 1], sm.hy[g][lxs[1]][lys[1] + 1]),
                                  make_float2(sm.hy[g][lxs[0]][lys[0]], sm.hy[g][lxs[1]][lys[1]]));
          X = __ffma2_rn(f2s(dtdy * p.pyh[pop]), dfy, X);
        }
        const int64_t e0 = (int64_t)pop * N + cell[0], e1 = (int64_t)pop * N + cell[1];
        const float2 d = make_float2(sm.ownd[g][o0], sm.ownd[g][o1]);
        float2 R;
        if constexpr (STAGE == kStage3) {
          const float2 f = make_float2(sm.ownv[g][o0], sm.ownv[g][o1]);
          R = __ffma2_rn(f2s(-sc.at32), X, __ffma2_rn(f2s(-sc.k3), d, f));
          const float2 a4 = __ffma2_rn(f2s(-sc.at42), X, __ffma2_rn(f2s(-sc.k4), d, f));
          const float2 af = __ffma2_rn(f2s(-sc.wt2), X, __ffma2_rn(f2s(-sc.kf), d, f));
          if (valid[0]) { R3[e0] = R.x; A4[e0] = a4.x; Af[e0] = af.x; }
          if (valid[1]) { R3[e1] = R.y; A4[e1] = a4.y; Af[e1] = af.y; }
        } else if constexpr (STAGE == kStage4) {
          R = __ffma2_rn(f2s(-sc.at43), X,
                         __ffma2_rn(f2s(-sc.a43e3), d, make_float2(a4v[0][g], a4v[1][g])));
          const float2 af = __ffma2_rn(f2s(-sc.wt3), X,
                                       __ffma2_rn(f2s(-sc.w3e3), d, make_float2(afv[0][g], afv[1][g])));
          if (valid[0]) { A4[e0] = R.x; Af[e0] = af.x; }
          if (valid[1]) { A4[e1] = R.y; Af[e1] = af.y; }
        } else {
          R = __ffma2_rn(f2s(-sc.wt4), X,
                         __ffma2_rn(f2s(-sc.w4e4), d, make_float2(afv[0][g], afv[1][g])));
          if (valid[0]) F[e0] = R.x;
          if (valid[1]) F[e1] = R.y;
        }
        accumulate2<DIM, QP, QC>(p, mom2, pop, R);
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
        float X = (dtdx * p.pxh[pop]) * (sm.hx[g][ly][lx + 1] - sm.hx[g][ly][lx]);
        if constexpr (DIM == 2)
          X = fmaf(dtdy * p.pyh[pop], sm.hy[g][lx][ly + 1] - sm.hy[g][lx][ly], X);
        const int64_t e = (int64_t)pop * N + cell[k];
        const float d = sm.ownd[g][o];
        float R;
        if constexpr (STAGE == kStage3) {
          const float f = sm.ownv[g][o];
          R = fmaf(-sc.at32, X, fmaf(-sc.k3, d, f));
          R3[e] = R;
          A4[e] = fmaf(-sc.at42, X, fmaf(-sc.k4, d, f));
          Af[e] = fmaf(-sc.wt2, X, fmaf(-sc.kf, d, f));
        } else if constexpr (STAGE == kStage4) {
          R = fmaf(-sc.at43, X, fmaf(-sc.a43e3, d, a4v[k][g]));
          A4[e] = R;
          Af[e] = fmaf(-sc.wt3, X, fmaf(-sc.w3e3, d, afv[k][g]));
        } else {
          R = fmaf(-sc.wt4, X, fmaf(-sc.w4e4, d, afv[k][g]));
          F[e] = R;
        }
        accumulate<DIM, QP, QC>(p, mom[k], pop, R);
      }
    }
    }
    __syncthreads();
  }
  if constexpr (CPT == 2) {
    mom[0] = lane(mom2, 0);
    mom[1] = lane(mom2, 1);
  }
  // ---- records of the stage's explicit parts (the next kernel relaxes them)
#pragma unroll
  for (int k = 0; k < CPT; ++k)
    if (valid[k]) finish_cell<DIM, QP, QC>(p, kchi_df, invDK_df, geo.prob, mom[k], rout, cell[k]);
}

template <int DIM, int QP, int QC, int STAGE, int VAR = 0>
__global__ void __launch_bounds__(TileCfg<DIM, VAR>::NT,
                                  DIM == 2 ? (STAGE == kStage3 ? 4 : 5)
                                           : (TileCfg<DIM, VAR>::NT >= 128 ? 5 : 8))
    mixed_stage_kernel(const __grid_constant__ DevParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  auto& sm = *reinterpret_cast<MixSmem<DIM, QP, QC, VAR, STAGE>*>(smraw);
  const Geo geo{p.nx, p.ny, 0, p.kchi, p.invDK, p.dtdx, p.dtdy, -1};
  mixed_tile<DIM, QP, QC, STAGE, VAR>(p, geo, blockIdx.x * TileCfg<DIM, VAR>::TX,
                                      blockIdx.y * TileCfg<DIM, VAR>::TY, sm);
}

template <int QP, int QC, int STAGE, int VAR>
__global__ void __launch_bounds__(TileCfg<1, VAR>::NT, 6)
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

// The record of F^n (after fdlb_init_riemann or fdlb_set_state): the same
// moment sums, in the same population order, as the final stage's.
template <int DIM, int QP, int QC>
__global__ void mixed_prep_kernel(const __grid_constant__ DevParams p) {
  using L = Lat<DIM, QP, QC>;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  const float* F = (const float*)p.F;
  MomentsF m = {};
  for (int pop = 0; pop < L::P; ++pop) accumulate<DIM, QP, QC>(p, m, pop, F[pop * p.N + c]);
  Geo geo{p.nx, p.ny, 0, p.kchi, p.invDK, p.dtdx, p.dtdy, -1};
  if (p.nprob > 0) {
    const int b = problem_of(p, c);
    geo.kchi = p.probs[b].kchi;
    geo.invDK = p.probs[b].invDK;
    geo.prob = b;
  }
  finish_cell<DIM, QP, QC>(p, df_of(geo.kchi), df_of(geo.invDK), geo.prob, m, p.erec[0], c);
}

template <int DIM, int QP, int QC, int VAR, int STAGE>
constexpr int smem_bytes() {
  return (int)sizeof(MixSmem<DIM, QP, QC, VAR, STAGE>);
}

template <int DIM, int QP, int QC>
int setup_t() {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mixed_stage_kernel<DIM, QP, QC, kStage3>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<DIM, QP, QC, 0, kStage3>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mixed_stage_kernel<DIM, QP, QC, kStage4>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<DIM, QP, QC, 0, kStage4>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mixed_stage_kernel<DIM, QP, QC, kFinal>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<DIM, QP, QC, 0, kFinal>());
  return (int)e;
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

template <int DIM, int QP, int QC>
int launch_t(const DevParams& p, int stage, cudaStream_t s) {
  if (stage == kPrep) {
    const int nt = 128;
    const int64_t nb = (p.N + nt - 1) / nt;
    mixed_prep_kernel<DIM, QP, QC><<<(unsigned)nb, nt, 0, s>>>(p);
    return (int)cudaGetLastError();
  }
  if constexpr (DIM == 1) {
    // 1-D problems pick their tile shape by length (single_1d_variant)
    switch (single_1d_variant(p.nx)) {
      case 1: return launch_tv<1, QP, QC, 1>(p, stage, s);
      case 3: return launch_tv<1, QP, QC, 3>(p, stage, s);
      case 4: return launch_tv<1, QP, QC, 4>(p, stage, s);
      default: return launch_tv<1, QP, QC, 0>(p, stage, s);
    }
  }
  return launch_tv<DIM, QP, QC, 0>(p, stage, s);
}

template <int QP, int QC, int VAR>
int launch_batch_v(const DevParams& p, int stage, cudaStream_t s) {
  using C = TileCfg<1, VAR>;
  const int grid = p.bgrid > 0 ? p.bgrid : 1;
  switch (stage) {
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
  if (stage == kPrep) {
    const int nt = 128;
    const int64_t nb = (p.N + nt - 1) / nt;
    mixed_prep_kernel<1, QP, QC><<<(unsigned)nb, nt, 0, s>>>(p);
    return (int)cudaGetLastError();
  }
  switch (p.variant) {
    case 1: return launch_batch_v<QP, QC, 1>(p, stage, s);
    case 2: return launch_batch_v<QP, QC, 2>(p, stage, s);
    default: return launch_batch_v<QP, QC, 0>(p, stage, s);
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

}  // namespace fdlb
