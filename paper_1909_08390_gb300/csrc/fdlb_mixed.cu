// fdlb_mixed.cu -- binary32 stage kernels of the IMEX step (FDLB_MIXED).
//
// Storage.  Every population of the state F^n is an unevaluated pair of
// binary32 values sh + sl with |sl| <= ulp(sh)/2 (about 48 significant
// bits).  The explicit parts of the stages are kept as binary32 low parts
// relative to sh (R3 = sh + r3l, A4' = sh + a4l, A_fin = sh + afl), small
// where the flow is smooth, so that their rounding is relative to the
// increment and not to the population.  (A binary32 copy of F rounded at
// every stage loses about 6e-8 of each population per stage; over thousands
// of steps that noise moves shocks and contacts far more than the 1e-5 the
// mixed path is held to.)
//
// Each stage kernel runs two passes over its tile:
//   pass 1, per group of populations: stage the advected values on the tile
//     and its 5-cell halo -- sh plus the binary32 low part the previous
//     kernel left for this stage (relative to one reference per population
//     and 2-D tile) --, march the MP-9 interface values (Sec. IV), form the
//     flux difference X and the stage's explicit parts (Eq. IMEX), store
//     them, and sum the moments of the stage's R (Eq. Moments_discrete);
//   pass 2, per own cell: n, u, T in binary64 from the moment sums (the
//     cancellation T = (e - j.u)/((D+K) n) included), the cell's equilibrium
//     factors (Eq. gExpanded) in binary32-pair arithmetic, and for every
//     population D = R - F_eq = (sh - Eh) + (low part - El), accurate to
//     its own size, and the low part of the relaxed value the next kernel
//     advects (Sec. III closed forms):
//       stage 3 leaves D3 and F3 - sh = r3l - a33 e3 D3,
//       stage 4 leaves D4 and F4 - sh = r4l - a44 e4 D4,
//       the final stage leaves the new state's D and F2 - sh = sl - (1 - c2) D
//       for the next step's stage 3.
// The relaxation is thus applied once per cell, by its owner, not on every
// staged copy of the halo, and no equilibrium data reach memory.
//
// Copies.  On 2-D grids whose rows hold a multiple of 4 cells, the staged
// tile and halo and the own cells' inputs arrive as 16-byte asynchronous
// copies (chunks of 4 cells, fdlb_tile.cuh), and pass 2 of a tile inside
// the grid streams its values through the then idle staging buffers, a ring
// of four chunks copied three steps ahead; elsewhere copies are per cell.
// Grids whose sides are multiples of the 16-cell tile, on lattices whose
// populations fill whole groups, run an instance compiled without the
// per-cell paths (FAST): unexecuted code in these kernels costs time.
//
// Moments: R3's and R4's are the binary64 per-cell sums of sh (mhi, left by
// the previous final stage) plus binary32 sums of their low parts; the final
// stage sums the new state's sh with error-free transformations (TwoSum and
// the fma product error) and its sl plainly, and stores the sums of sh.
//
// Arrays per population and step (binary32): stage 3 stages sh and fa, reads
// D and sl of its cells, writes r3l, a4l, afl, then re-reads sh and r3l and
// writes D and fb; stage 4 stages sh and fb, reads D, a4l, afl, writes a4l
// (now R4's low part) and afl, then re-reads sh and a4l and writes D and fc;
// the final stage stages sh and fc, reads D, afl and sh, writes the next
// state nh, nl, then re-reads them and writes D and fa.
#include <cstddef>

#include "fdlb_device.cuh"

namespace fdlb {
namespace {

// 16-byte asynchronous copy, L2 only (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_2() { asm volatile("cp.async.wait_group 2;\n" ::: "memory"); }

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

// Equilibrium factors of a cell (Eq. gExpanded) from binary64 n, u, T, in
// binary32-pair arithmetic: phi^eq(kx, ky) = A[kx] B[ky] (1-D: A[k]) with
// A = n g_x, B = g_y; chi^eq(qx, qy) = A[qx] C B[qy] (1-D: C A[q]) with C =
// (D+K-d) T when Qchi = Qphi, else Hx[qx] Hy[qy] (1-D: H[q]) with Hx =
// C n h_x, Hy = h_y.
template <int DIM, int QP, int QC>
struct EqFac {
  static constexpr bool kSame = QP == QC;
  DF A[QP], B[DIM == 2 ? QP : 1], C;
  DF Hx[kSame ? 1 : QC], Hy[(kSame || DIM == 1) ? 1 : QC];
};

template <int DIM, int QP, int QC>
__device__ __forceinline__ void eq_factors(const DevParams& p, double kchi, double n, double ux,
                                           double uy, double T, EqFac<DIM, QP, QC>& f) {
  const DF dn = df_of(n), dux = df_of(ux), dT = df_of(T), one{1.0f, 0.0f};
  axis_g_df<QP>(p.wHph, p.wHpl, dux, dT, dn, f.A);
  if constexpr (DIM == 2) axis_g_df<QP>(p.wHph, p.wHpl, df_of(uy), dT, one, f.B);
  f.C = df_mul(df_of(kchi), dT);
  if constexpr (!EqFac<DIM, QP, QC>::kSame) {
    axis_g_df<QC>(p.wHch, p.wHcl, dux, dT, df_mul(f.C, dn), f.Hx);
    if constexpr (DIM == 2) axis_g_df<QC>(p.wHch, p.wHcl, df_of(uy), dT, one, f.Hy);
  }
}

// The populations of a cell in rows of at most kMaxRow that share one
// factor of their equilibrium: 2-D, the phi rows ky and the chi rows qy
// (first population, length); 1-D, the phi and the chi populations.
template <int DIM, int QP, int QC>
struct EqRows {
  static constexpr int R = DIM == 2 ? QP + QC : 2;
  __host__ __device__ static constexpr int len(int r) { return DIM == 2 ? (r < QP ? QP : QC) : (r == 0 ? QP : QC); }
  __host__ __device__ static constexpr int first(int r) {
    return DIM == 2 ? (r < QP ? r * QP : QP * QP + (r - QP) * QC) : (r == 0 ? 0 : QP);
  }
};
constexpr int kMaxRow = 8;

// The row factor of row r and the equilibrium pair of its j-th population.
template <int DIM, int QP, int QC>
__device__ __forceinline__ DF eq_row_factor(const EqFac<DIM, QP, QC>& f, int r) {
  if constexpr (DIM == 2) {
    if (r < QP) return f.B[r];
    if constexpr (EqFac<DIM, QP, QC>::kSame) return df_mul(f.C, f.B[r - QP]);
    else return f.Hy[r - QP];
  } else {
    return f.C;
  }
}
template <int DIM, int QP, int QC>
__device__ __forceinline__ DF eq_in_row(const EqFac<DIM, QP, QC>& f, int r, DF rowf, int j) {
  if constexpr (DIM == 2) {
    if (r < QP) return pmul(f.A[j], rowf);
    if constexpr (EqFac<DIM, QP, QC>::kSame) return pmul(f.A[j], rowf);
    else return pmul(f.Hx[j], rowf);
  } else {
    if (r == 0) return f.A[j];
    if constexpr (EqFac<DIM, QP, QC>::kSame) return pmul(rowf, f.A[j]);
    else return f.Hx[j];
  }
}

// Pass 2 of a cell: its moment sums (binary64) -> validity flags, n, u and
// T = (e - j.u)/((D+K) n) (Eq. Moments_discrete and the temperature
// definition) in binary64, the equilibrium factors, and for every population
// D = (a - Eh) + (b - El) of the value R = a + b (a = sh, b its low part) and
// the low part b - kd D of the relaxed value R - kd D: D to dm, the low part
// to fout.
template <int DIM, int QP, int QC>
__device__ __forceinline__ void relax_cell(const DevParams& p, double kchi, double invDK, int prob,
                                           double n, double jx, double jy, double e,
                                           const float* __restrict__ ain,
                                           const float* __restrict__ bin, float kd,
                                           float* __restrict__ fout, int64_t cell) {
  const double inv_n = 1.0 / n;
  const double ux = jx * inv_n;
  const double uy = DIM == 2 ? jy * inv_n : 0.0;
  const double T = (e - fma(jx, ux, jy * uy)) * inv_n * invDK;
  const bool ok = n > 0.0 && T > 0.0 && isfinite(n) && isfinite(T) && isfinite(ux) && isfinite(uy);
  if (!ok) {
    atomicOr(p.status, 1u);
    if (prob >= 0) atomicOr(&p.pstatus[prob], 1u);
  }
  EqFac<DIM, QP, QC> fac;
  eq_factors<DIM, QP, QC>(p, kchi, n, ux, uy, T, fac);
  const int64_t N = p.N;
  using RW = EqRows<DIM, QP, QC>;
  // row by row, the next row's values loaded before this row is computed
  float ca[kMaxRow], cb[kMaxRow], na[kMaxRow], nb[kMaxRow];
  auto load = [&](int r, float (&a)[kMaxRow], float (&b)[kMaxRow]) {
#pragma unroll
    for (int j = 0; j < kMaxRow; ++j)
      if (j < RW::len(r)) {
        const int64_t i = (int64_t)(RW::first(r) + j) * N + cell;
        a[j] = ain[i];
        b[j] = bin[i];
      }
  };
  load(0, ca, cb);
#pragma unroll
  for (int r = 0; r < RW::R; ++r) {
    if (r + 1 < RW::R) load(r + 1, na, nb);
    const DF rowf = eq_row_factor<DIM, QP, QC>(fac, r);
#pragma unroll
    for (int j = 0; j < kMaxRow; ++j)
      if (j < RW::len(r)) {
        const DF E = eq_in_row<DIM, QP, QC>(fac, r, rowf, j);
        const int64_t i = (int64_t)(RW::first(r) + j) * N + cell;
        const float d = __fadd_rn(__fsub_rn(ca[j], E.hi), __fsub_rn(cb[j], E.lo));
        p.dm[i] = d;
        fout[i] = fmaf(-kd, d, cb[j]);
      }
#pragma unroll
    for (int j = 0; j < kMaxRow; ++j) {
      ca[j] = na[j];
      cb[j] = nb[j];
    }
  }
}

// Pass 2 of a 2-D tile wholly inside a grid of 16-byte aligned rows: the
// cells' values of R (a + b) stream through a ring of NB shared buffers, one
// chunk (a row of the cell's equilibrium, for half of the tile's cells: the
// cells tid, then tid + NT) per step, copied 16 bytes at a time three steps
// ahead; each thread computes its own cell of every chunk, with the same
// arithmetic as relax_cell.
// a[k] for a k known only at run time, by selects (no local memory)
template <int Q>
__device__ __forceinline__ DF pick_df(const DF (&a)[Q], int k) {
  DF v = a[0];
#pragma unroll
  for (int i = 1; i < Q; ++i)
    if (k == i) v = a[i];
  return v;
}

template <int DIM, int QP, int QC, int TX, int TY, int NT>
__device__ __forceinline__ void relax_tile_streamed(const DevParams& p, double kchi, double invDK,
                                                    int prob, const double (&mom)[2][4],
                                                    int64_t N, int64_t cell0, int nx,
                                                    const float* __restrict__ ain,
                                                    const float* __restrict__ bin, float kd,
                                                    float* __restrict__ fout, float* __restrict__ ring) {
  using RW = EqRows<DIM, QP, QC>;
  constexpr int HALF = NT;                 // cells of one chunk
  constexpr int CS = 2 * kMaxRow * HALF;   // floats of one chunk buffer
  constexpr int NB = 4;
  constexpr int NS = 2 * RW::R;            // steps: two halves x rows
  static_assert(TX * TY == 2 * NT && HALF % TX == 0, "two halves of whole rows");
  const int tid = threadIdx.x;
  // chunk s: half s / R, row s % R; slot (j, a, c) at (j * 2 + a) * HALF + c
  auto issue = [&](int s) {
    if (s < NS) {
      const int k = s / RW::R, r = s % RW::R;
      float* buf = ring + (s % NB) * CS;
      constexpr int PER = 2 * kMaxRow * HALF / 4;  // 16-byte chunks
#pragma unroll
      for (int i = 0; i < (PER + NT - 1) / NT; ++i) {
        const int q = tid + i * NT;
        if (q < PER) {
          const int ja = q / (HALF / 4), c4 = (q % (HALF / 4)) * 4;
          const int j = ja >> 1, a = ja & 1;
          if (j < RW::len(r)) {
            const int ci = k * HALF + c4;  // tile cell of the chunk's first cell
            const int64_t g = (int64_t)(RW::first(r) + j) * N + cell0 + (int64_t)(ci / TX) * nx + ci % TX;
            cp_async16(buf + ja * HALF + c4, (a ? bin : ain) + g);
          }
        }
      }
    }
    cp_async_commit();
  };
  issue(0);
  issue(1);
  issue(2);
  EqFac<DIM, QP, QC> fac;
  int64_t mycell = 0;
#pragma unroll 1
  for (int s = 0; s < NS; ++s) {
    const int k = s / RW::R, r = s % RW::R;
    if (r == 0) {
      const double n = mom[k][0], jx = mom[k][1], jy = mom[k][2], e = mom[k][3];
      const double inv_n = 1.0 / n;
      const double ux = jx * inv_n;
      const double uy = DIM == 2 ? jy * inv_n : 0.0;
      const double T = (e - fma(jx, ux, jy * uy)) * inv_n * invDK;
      const bool ok = n > 0.0 && T > 0.0 && isfinite(n) && isfinite(T) && isfinite(ux) && isfinite(uy);
      if (!ok) {
        atomicOr(p.status, 1u);
        if (prob >= 0) atomicOr(&p.pstatus[prob], 1u);
      }
      eq_factors<DIM, QP, QC>(p, kchi, n, ux, uy, T, fac);
      const int ci = k * HALF + tid;
      mycell = cell0 + (int64_t)(ci / TX) * nx + ci % TX;
    }
    cp_async_wait_2();
    __syncthreads();
    const float* buf = ring + (s % NB) * CS;
    // one copy of the row body: the row factor is picked at run time (the
    // same factors and products as eq_row_factor, eq_in_row)
    using FAC = EqFac<DIM, QP, QC>;
    DF rowf;
    if (r < QP) rowf = pick_df<QP>(fac.B, r);
    else if constexpr (FAC::kSame) rowf = df_mul(fac.C, pick_df<QP>(fac.B, r - QP));
    else rowf = pick_df<QC>(fac.Hy, r - QP);
    const int len = RW::len(r), first = RW::first(r);
    const bool phi_row = r < QP;
#pragma unroll
    for (int j = 0; j < kMaxRow; ++j)
      if (j < len) {
        DF colf;
        if constexpr (FAC::kSame) colf = fac.A[j < QP ? j : 0];
        else colf = phi_row ? fac.A[j < QP ? j : 0] : fac.Hx[j < QC ? j : 0];
        const DF E = pmul(colf, rowf);
        const float a = buf[(2 * j) * HALF + tid], b = buf[(2 * j + 1) * HALF + tid];
        const int64_t i = (int64_t)(first + j) * N + mycell;
        const float d = __fadd_rn(__fsub_rn(a, E.hi), __fsub_rn(b, E.lo));
        p.dm[i] = d;
        fout[i] = fmaf(-kd, d, b);
      }
    issue(s + 3);
  }
  cp_async_wait_all();
  __syncthreads();
}

// Plain binary32 moment sums of low parts, one cell or two (packed lanes).
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

template <int DIM, int QP, int QC, int VAR, int STAGE>
struct MixSmem {
  using C = TileCfg<DIM, VAR>;
  // own-cell inputs of pass 1: D and the low parts the stage updates
  // (stage 3: sl; stage 4: a4l, afl; final: afl, sh)
  static constexpr int NOWN = STAGE == kStage3 ? 2 : 3;
  static constexpr int SXH = C::TX + 2 * H;             // staged columns
  static constexpr int SX = SXH + (DIM == 2 ? 1 : 0);   // tile row pitch
  static constexpr int SY = DIM == 2 ? C::TY + 2 * H : 1;
  // staged cells: tile + halo without the 2-D corner blocks (staged_pos)
  static constexpr int NSC = DIM == 2 ? C::TY * SXH + 2 * H * C::TX : SXH;
  // 2-D grids whose rows hold a multiple of 4 cells land whole 16-byte
  // chunks: the H rows above and below the tile (its columns), and the
  // tile's rows from 8 columns left to 8 columns right of it (the 5-cell
  // halos rounded out to chunks); other tiles land cell by cell
  static constexpr int NCL = DIM == 2 && C::TX % 4 == 0 ? 2 * H * C::TX + C::TY * (C::TX + 16) : 0;
  static constexpr int NRAW = NCL > NSC ? NCL : NSC;
  float rawh[C::G][NRAW];              // sh of the staged cells, as loaded
  float rawf[C::G][NRAW];              // the advected low parts, as loaded
  float tile[C::G][SY][SX];            // advected values - ref
  // 2-D: flux differences of the cells along x and y (mp9_march_delta_fp32);
  // 1-D: interface values along x.  Rows of TX + 1 (TY + 1) floats: the odd
  // pitch keeps the march's column-wise writes free of bank conflicts.
  float hx[C::G][C::TY][C::TX + 1];
  float hy[DIM == 2 ? C::G : 1][DIM == 2 ? C::TX : 1][DIM == 2 ? C::TY + 1 : 1];
  // dt p / ds per population as binary32 pairs: (x hi, x lo, y hi, y lo)
  float4 coef[Lat<DIM, QP, QC>::P];
  float own[NOWN][C::G][C::TX * C::TY];
};

// One tile of one stage.  Ends with every thread past its last use of the
// shared memory, so a persistent CTA may start its next tile at once.
// FAST: a 2-D grid whose sides are multiples of the tile's and whose
// populations fill whole groups (every tile full, every row 16-byte
// aligned), compiled without the per-cell copy and relaxation paths (the
// kernels are sensitive to code size).
template <int DIM, int QP, int QC, int STAGE, int VAR, bool FAST = false>
__device__ __forceinline__ void mixed_tile(const DevParams& p, const Geo& geo, int x0, int y0,
                                           MixSmem<DIM, QP, QC, VAR, STAGE>& sm) {
  using C = TileCfg<DIM, VAR>;
  using L = Lat<DIM, QP, QC>;
  using M = MixSmem<DIM, QP, QC, VAR, STAGE>;
  constexpr int TX = C::TX, TY = C::TY, NT = C::NT, G = C::G, SEG = C::SEG;
  constexpr int SX = M::SX, NSC = M::NSC;
  constexpr int CELLS = TX * TY;
  constexpr int CPT = (CELLS + NT - 1) / NT;
  constexpr int NSEG = (TX + 1) / SEG;
  static_assert(NSEG * SEG == TX + 1, "segments tile the line");
  constexpr int NLINE = DIM == 2 ? TX + TY : 1;
  static_assert(G * NLINE * NSEG == NT, "one march task per thread");
  constexpr int J = (NSC + NT - 1) / NT;  // staged cells per thread
  constexpr int NG = (L::P + G - 1) / G;

  const float* __restrict__ const Sh = p.sh;
  // the advected low parts: F2 - sh (stage 3), F3 - sh (stage 4), F4 - sh
  // (final stage), left by the previous kernel's pass 2
  const float* __restrict__ const fin = STAGE == kStage3 ? p.fa : (STAGE == kStage4 ? p.fb : p.fc);
  const int tid = threadIdx.x;
  const int64_t N = p.N;

  // chunked landing (16-byte copies) for 2-D grids whose rows, and so all
  // chunk addresses, are 16-byte aligned; else cell by cell
  constexpr bool kCh = M::NCL > 0;
  constexpr bool kFast = FAST && DIM == 2 && kCh && L::P % G == 0;
  static_assert(!FAST || kFast, "FAST needs 2-D chunked tiles and whole groups");
  const bool chunked = kFast || (kCh && (geo.nx % 4) == 0 && (geo.base % 4) == 0);
  // this thread's staged cells: tile offset and landing slot (-1: none);
  // cell by cell, slot e holds staged cell e, and 1-D keeps its offset from
  // geo.base (2-D grids landed cell by cell recompute it)
  int soff[J], loff[J], goff1[DIM == 1 ? J : 1];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int e = tid + j * NT;
    int r, c;
    staged_pos(e, DIM, TX, TY, r, c);
    soff[j] = r * SX + c;
    loff[j] = -1;
    if (e < NSC) {
      loff[j] = e;
      if constexpr (DIM == 1) goff1[j] = wrap_or_clamp(x0 - H + c, geo.nx, p.bc);
      if (chunked) loff[j] = chunk_slot(r, c, TX, TY, x0, geo.nx, p.bc);
    }
  }
  // the thread's chunks q = tid, tid + NT (chunk_offset; -1: not copied)
  constexpr int NCHK = M::NCL / 4;
  static_assert(!kCh || NCHK <= 2 * NT, "two chunks per thread at most");
  int go[2] = {-1, -1};
  if constexpr (kCh) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
      if (chunked && tid + i * NT < NCHK)
        go[i] = chunk_offset(tid + i * NT, TX, TY, x0, y0, geo.nx, geo.ny, p.bc);
  }
  // own cells of this thread: tid + k NT (coalesced in both passes); a slot
  // past the tile's cells takes cell 0's indices (its lane computes on them
  // and stores nothing), so every shared-memory index stays inside its array
  int lxs[CPT], lys[CPT];
  int64_t cell[CPT];
  bool valid[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    const int ci = tid + k * NT;
    const int c = ci < CELLS ? ci : 0;
    lxs[k] = c % TX;
    lys[k] = c / TX;
    valid[k] = (ci < CELLS) && (x0 + lxs[k] < geo.nx) && (y0 + lys[k] < geo.ny);
    cell[k] = geo.base + (int64_t)(y0 + lys[k]) * geo.nx + (x0 + lxs[k]);
  }
  // moment sums: stages 3 and 4 sum the low parts of R3, R4 plainly; the
  // final stage sums the new sh error-free (mom) and the new sl plainly
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
  // coefficients that multiply advection terms of the size of the
  // populations' variation, as binary32 pairs: dt p / ds (a rounded speed
  // would shift every wave coherently) and the explicit weights wt2, wt3,
  // wt4 (1/6, 1/6, 2/3, whose rounded sum misses 1)
  const float wtl = STAGE == kStage3 ? (float)(p.sc.wt2 - (double)sc.wt2)
                  : STAGE == kStage4 ? (float)(p.sc.wt3 - (double)sc.wt3)
                                     : (float)(p.sc.wt4 - (double)sc.wt4);
  {
    const DF dtdx_df = df_of(geo.dtdx), dtdy_df = df_of(geo.dtdy);
    // dt p / ds of every population along x and y, once per tile (the first
    // barrier of the group loop orders it before pass 1); 2-D takes |.| (the
    // flux differences of the 2-D march carry the velocity's sign)
    for (int pop = tid; pop < L::P; pop += NT) {
      DF cx = df_mul(dtdx_df, DF{p.pxh[pop], p.pxl[pop]});
      DF cy = DIM == 2 ? df_mul(dtdy_df, DF{p.pyh[pop], p.pyl[pop]}) : DF{0.0f, 0.0f};
      if (DIM == 2 && cx.hi < 0.0f) cx = df_neg(cx);
      if (DIM == 2 && cy.hi < 0.0f) cy = df_neg(cy);
      sm.coef[pop] = make_float4(cx.hi, cx.lo, cy.hi, cy.lo);
    }
  }
  // the reference value of each population on a 2-D tile: sh at the tile's
  // first cell.  1-D tiles take none, so that a 1-D problem gives the same
  // bits whatever its tiling (batches and single problems use different
  // tile lengths).
  const int64_t cref = geo.base + (int64_t)y0 * geo.nx + x0;

  const int tg = tid / (NLINE * NSEG);  // the thread's population in a group (march)
  const int tline = (tid / NSEG) % NLINE;
  // landed cell by cell, each thread copies, and later reads, only its own
  // staged cells, so its own wait on the copies orders them; chunks are read
  // by other threads, so a barrier follows the wait
  float refv[G];
  auto prefetch = [&](int gfirst) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int pop = gfirst + g;
      if (pop >= L::P) break;
      const float* __restrict__ srch = Sh + (int64_t)pop * N + geo.base;
      const float* __restrict__ srcf = fin + (int64_t)pop * N + geo.base;
      if (kFast || (kCh && chunked)) {
#pragma unroll
        for (int i = 0; i < 2; ++i)
          if (go[i] >= 0) {
            cp_async16(&sm.rawh[g][4 * (tid + i * NT)], srch + go[i]);
            cp_async16(&sm.rawf[g][4 * (tid + i * NT)], srcf + go[i]);
          }
      } else if constexpr (!kFast) {
#pragma unroll
        for (int j = 0; j < J; ++j)
          if (loff[j] >= 0) {
            int o;
            if constexpr (DIM == 1) {
              o = goff1[j];
            } else {
              int r, c;
              staged_pos(tid + j * NT, DIM, TX, TY, r, c);
              o = wrap_or_clamp(y0 - H + r, geo.ny, p.bc) * geo.nx +
                  wrap_or_clamp(x0 - H + c, geo.nx, p.bc);
            }
            cp_async(&sm.rawh[g][loff[j]], srch + o);
            cp_async(&sm.rawf[g][loff[j]], srcf + o);
          }
      }
      refv[g] = DIM == 2 ? Sh[(int64_t)pop * N + cref] : 0.0f;
    }
    cp_async_commit();
  };
  // the own cells' inputs of pass 1 for group gfirst, copied asynchronously
  // into sm.own (each thread copies and reads only its own cells' slots):
  // D of the stage's input and the low parts it updates (stage 3: sl;
  // stage 4: a4l, afl; final: afl, sh)
  // A 2-D tile wholly inside a grid of 16-byte aligned rows copies them as
  // 16-byte chunks of 4 cells, any thread any chunk (the barrier before
  // pass 1 orders them).
  const bool own16 = kFast || (DIM == 2 && TX % 4 == 0 && (geo.nx % 4) == 0 && (geo.base % 4) == 0 &&
                     x0 + TX <= geo.nx && y0 + TY <= geo.ny);
  auto prefetch_own = [&](int gfirst) {
    const float* const src[3] = {p.dm, STAGE == kStage3 ? p.sl : (STAGE == kStage4 ? p.a4l : p.afl),
                                 STAGE == kStage4 ? p.afl : Sh};
    if constexpr (DIM == 2) {
      if (kFast || (own16 && gfirst + G <= L::P)) {
        constexpr int CH = CELLS / 4;  // chunks per population and array
        constexpr int NCH = M::NOWN * G * CH;
        static_assert(NCH % NT == 0, "whole chunks per thread");
#pragma unroll
        for (int i = 0; i < NCH / NT; ++i) {
          const int q = tid + i * NT;
          const int a = q / (G * CH), g = (q / CH) % G, cq = q % CH;
          const int row = cq / (TX / 4), c4 = (cq % (TX / 4)) * 4;
          const float* sa = a == 0 ? src[0] : (a == 1 ? src[1] : src[M::NOWN - 1]);
          cp_async16(&sm.own[a][g][row * TX + c4],
                     sa + (int64_t)(gfirst + g) * N + geo.base + (int64_t)(y0 + row) * geo.nx + x0 + c4);
        }
        cp_async_commit();
        return;
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int pop = gfirst + g;
      if (pop >= L::P) break;
#pragma unroll
      for (int k = 0; k < CPT; ++k)
        if (valid[k]) {
          const int64_t e = (int64_t)pop * N + cell[k];
#pragma unroll
          for (int a = 0; a < M::NOWN; ++a) cp_async(&sm.own[a][g][tid + k * NT], src[a] + e);
        }
    }
    cp_async_commit();
  };
  // copy groups in flight: the staged values of group gi + 1 are committed
  // after the own inputs of group gi, and the own inputs of group gi + 1
  // after pass 1 of group gi, so that waiting for all but the newest group
  // completes the data needed next
  prefetch(0);
  prefetch_own(0);
  for (int gi = 0; gi < NG; ++gi) {
    const int g0 = gi * G;  // first population of the group
    // ---- stage the group: advected values - ref on tile + halo (chunks
    // land from other threads: group 0's before this barrier, later groups'
    // before the previous group's last barrier)
    cp_async_wait_1();
    if (kCh && gi == 0) __syncthreads();
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int pop = g0 + g;
      if (pop >= L::P) break;
      const float ref = refv[g];
#pragma unroll
      for (int j = 0; j < J; ++j)
        if (loff[j] >= 0) {
          const int e = loff[j];
          (&sm.tile[g][0][0])[soff[j]] = __fadd_rn(__fsub_rn(sm.rawh[g][e], ref), sm.rawf[g][e]);
        }
    }
    __syncthreads();
    if (gi + 1 < NG) prefetch((gi + 1) * G);  // overlaps the march and pass 1
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
    // the own inputs of this group (the newest group in flight is the next
    // group's staged values, if any)
    if (gi + 1 < NG) cp_async_wait_1();
    else cp_async_wait_all();
    __syncthreads();
    // ---- flux difference and explicit parts of the own cells (pass 1)
    auto xflux = [&](int pop, int lx, int ly) {
      const float4 cf = sm.coef[pop];
      if constexpr (DIM == 2) {
        const float dx = sm.hx[pop - g0][ly][lx], dy = sm.hy[pop - g0][lx][ly];
        const float X = fmaf(cf.x, dx, __fmul_rn(cf.y, dx));
        return fmaf(cf.z, dy, fmaf(cf.w, dy, X));
      } else {
        const float dfx = __fsub_rn(sm.hx[pop - g0][ly][lx + 1], sm.hx[pop - g0][ly][lx]);
        return fmaf(cf.x, dfx, __fmul_rn(cf.y, dfx));
      }
    };
    if constexpr (CPT == 2) {
      // the thread's two cells in lockstep, as packed binary32 pairs (lane 1
      // of a cell outside the grid computes on unused values, never stored)
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int pop = g0 + g;
        if (pop >= L::P) break;
        const float2 X = make_float2(xflux(pop, lxs[0], lys[0]), xflux(pop, lxs[1], lys[1]));
        const int64_t e0 = (int64_t)pop * N + cell[0], e1 = (int64_t)pop * N + cell[1];
        auto put = [&](float* __restrict__ a, float2 v) {
          if (valid[0]) a[e0] = v.x;
          if (valid[1]) a[e1] = v.y;
        };
        const float2 d = make_float2(sm.own[0][g][tid], sm.own[0][g][tid + NT]);
        const float2 w1 = make_float2(sm.own[1][g][tid], sm.own[1][g][tid + NT]);
        if constexpr (STAGE == kStage3) {
          const float2 r3 = __fadd2_rn(w1, __ffma2_rn(f2s(-sc.at32), X, __fmul2_rn(f2s(-sc.k3), d)));
          const float2 a4 = __fadd2_rn(w1, __ffma2_rn(f2s(-sc.at42), X, __fmul2_rn(f2s(-sc.k4), d)));
          const float2 af = __fadd2_rn(
              w1, __ffma2_rn(f2s(-sc.wt2), X, __ffma2_rn(f2s(-wtl), X, __fmul2_rn(f2s(-sc.kf), d))));
          put(p.r3l, r3);
          put(p.a4l, a4);
          put(p.afl, af);
          accum_low2<DIM, QP, QC>(p, lm2, pop, r3);
        } else if constexpr (STAGE == kStage4) {
          const float2 w2 = make_float2(sm.own[M::NOWN - 1][g][tid], sm.own[M::NOWN - 1][g][tid + NT]);
          const float2 r4 = __ffma2_rn(f2s(-sc.at43), X, __ffma2_rn(f2s(-sc.a43e3), d, w1));
          const float2 af = __ffma2_rn(f2s(-sc.wt3), X,
                                       __ffma2_rn(f2s(-wtl), X, __ffma2_rn(f2s(-sc.w3e3), d, w2)));
          put(p.a4l, r4);
          put(p.afl, af);
          accum_low2<DIM, QP, QC>(p, lm2, pop, r4);
        } else {
          // F^{n+1} = sh + t with t = afl - w4 e4 D4 - wt4 X4, renormalised by
          // TwoSum into the next buffer
          const float2 a = make_float2(sm.own[M::NOWN - 1][g][tid],
                                       sm.own[M::NOWN - 1][g][tid + NT]);  // sh
          const float2 t = __ffma2_rn(f2s(-sc.wt4), X,
                                      __ffma2_rn(f2s(-wtl), X, __ffma2_rn(f2s(-sc.w4e4), d, w1)));
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
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int pop = g0 + g;
          if (pop >= L::P) break;
          const float X = xflux(pop, lxs[k], lys[k]);
          const int64_t e = (int64_t)pop * N + cell[k];
          const float d = sm.own[0][g][tid + k * NT], w1 = sm.own[1][g][tid + k * NT];
          if constexpr (STAGE == kStage3) {
            const float r3 = __fadd_rn(w1, fmaf(-sc.at32, X, __fmul_rn(-sc.k3, d)));
            p.r3l[e] = r3;
            p.a4l[e] = __fadd_rn(w1, fmaf(-sc.at42, X, __fmul_rn(-sc.k4, d)));
            p.afl[e] = __fadd_rn(w1, fmaf(-sc.wt2, X, fmaf(-wtl, X, __fmul_rn(-sc.kf, d))));
            accum_low<DIM, QP, QC>(p, lm[k], pop, r3);
          } else if constexpr (STAGE == kStage4) {
            const float r4 = fmaf(-sc.at43, X, fmaf(-sc.a43e3, d, w1));
            p.a4l[e] = r4;
            p.afl[e] = fmaf(-sc.wt3, X,
                            fmaf(-wtl, X, fmaf(-sc.w3e3, d, sm.own[M::NOWN - 1][g][tid + k * NT])));
            accum_low<DIM, QP, QC>(p, lm[k], pop, r4);
          } else {
            const float t = fmaf(-sc.wt4, X, fmaf(-wtl, X, fmaf(-sc.w4e4, d, w1)));
            const float a = sm.own[M::NOWN - 1][g][tid + k * NT];
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
    // the next group's staged copies, the only ones in flight, complete
    // before the barrier
    if constexpr (kCh) cp_async_wait_all();
    __syncthreads();
    if (gi + 1 < NG) prefetch_own((gi + 1) * G);
  }
  if constexpr (CPT == 2) {
    lm[0] = MomL{lm2.n.x, lm2.jx.x, lm2.jy.x, lm2.e.x};
    lm[1] = MomL{lm2.n.y, lm2.jx.y, lm2.jy.y, lm2.e.y};
    mom[0] = lane(mom2, 0);
    mom[1] = lane(mom2, 1);
  }
  // ---- pass 2, per own cell: binary64 moments of R3, R4 (or of the new
  // state), its equilibrium, D and the low part the next kernel advects
  const float kd = STAGE == kStage3 ? sc.a33e3
                 : STAGE == kStage4 ? sc.a44e4
                                    : (float)(1.0 - p.sc.c2);
  const float* __restrict__ const ain = STAGE == kFinal ? p.nh : Sh;
  const float* __restrict__ const bin = STAGE == kStage3 ? p.r3l : (STAGE == kStage4 ? p.a4l : p.nl);
  float* __restrict__ const fout = STAGE == kStage3 ? p.fb : (STAGE == kStage4 ? p.fc : p.fa);
  if constexpr (DIM == 2 && CPT == 2 && TX * TY == 2 * NT) {
    if (kFast || own16) {
      double mm[2][4];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
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
        mm[k][0] = mh[0] + (double)lm[k].n;
        mm[k][1] = mh[1] + (double)lm[k].jx;
        mm[k][2] = mh[2] + (double)lm[k].jy;
        mm[k][3] = mh[3] + (double)lm[k].e;
      }
      // the ring takes the staging buffers, rawh (offset 0) up to coef,
      // free once pass 1 has passed its last barrier
      static_assert(sizeof(float) * 4 * 2 * kMaxRow * NT <= offsetof(M, coef),
                    "the ring fits in the staging buffers");
      relax_tile_streamed<DIM, QP, QC, TX, TY, NT>(p, geo.kchi, geo.invDK, geo.prob, mm, N,
                                                   geo.base + (int64_t)y0 * geo.nx + x0, geo.nx,
                                                   ain, bin, kd, fout, &sm.rawh[0][0]);
      return;
    }
  }
  // other tiles, cell by cell
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
    relax_cell<DIM, QP, QC>(p, geo.kchi, geo.invDK, geo.prob, mh[0] + (double)lm[k].n,
                            mh[1] + (double)lm[k].jx, mh[2] + (double)lm[k].jy,
                            mh[3] + (double)lm[k].e, ain, bin, kd, fout, c);
  }
}

template <int DIM, int QP, int QC, int STAGE, int VAR = 0, bool FAST = false>
__global__ void __launch_bounds__(TileCfg<DIM, VAR>::NT,
                                  DIM == 2 ? 4 : (TileCfg<DIM, VAR>::NT >= 128 ? 5 : 8))
    mixed_stage_kernel(const __grid_constant__ DevParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  auto& sm = *reinterpret_cast<MixSmem<DIM, QP, QC, VAR, STAGE>*>(smraw);
  const Geo geo{p.nx, p.ny, 0, p.kchi, p.invDK, p.dtdx, p.dtdy, -1};
  mixed_tile<DIM, QP, QC, STAGE, VAR, FAST>(p, geo, blockIdx.x * TileCfg<DIM, VAR>::TX,
                                            blockIdx.y * TileCfg<DIM, VAR>::TY, sm);
}

// whether a lattice has a FAST instance: 2-D, populations in whole groups
template <int DIM, int QP, int QC>
constexpr bool fast_lattice() {
  return DIM == 2 && (QP * QP + QC * QC) % TileCfg<2, 0>::G == 0;
}

// (255-cell tiles carry two cells per thread: 3 CTAs per SM keep their
// registers unspilled)
template <int QP, int QC, int STAGE, int VAR>
__global__ void __launch_bounds__(TileCfg<1, VAR>::NT, VAR == 2 ? 3 : 5)
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

// After fdlb_init_riemann or fdlb_set_state: mhi, D and F2 - sh of the
// state, with the final stage's sums in the final stage's population order
// (so that a state set from a copy continues bit for bit).
template <int DIM, int QP, int QC>
__global__ void mixed_prep_kernel(const __grid_constant__ DevParams p) {
  using L = Lat<DIM, QP, QC>;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.N) return;
  MomentsF m = {};
  MomL lm = {};
  for (int pop = 0; pop < L::P; ++pop) {
    accumulate<DIM, QP, QC>(p, m, pop, p.sh[pop * p.N + c]);
    accum_low<DIM, QP, QC>(p, lm, pop, p.sl[pop * p.N + c]);
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
  relax_cell<DIM, QP, QC>(p, geo.kchi, geo.invDK, geo.prob, mh.n + (double)lm.n,
                          mh.jx + (double)lm.jx, mh.jy + (double)lm.jy, mh.e + (double)lm.e, p.sh,
                          p.sl, (float)(1.0 - p.sc.c2), p.fa, c);
}

template <int DIM, int QP, int QC, int VAR, int STAGE>
constexpr int smem_bytes() {
  return (int)sizeof(MixSmem<DIM, QP, QC, VAR, STAGE>);
}

template <int DIM, int QP, int QC, int VAR, bool FAST = false>
int setup_tv() {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mixed_stage_kernel<DIM, QP, QC, kStage3, VAR, FAST>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<DIM, QP, QC, VAR, kStage3>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mixed_stage_kernel<DIM, QP, QC, kStage4, VAR, FAST>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<DIM, QP, QC, VAR, kStage4>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mixed_stage_kernel<DIM, QP, QC, kFinal, VAR, FAST>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_bytes<DIM, QP, QC, VAR, kFinal>());
  return (int)e;
}

template <int DIM, int QP, int QC>
int setup_t() {
  int e = setup_tv<DIM, QP, QC, 0>();
  if constexpr (fast_lattice<DIM, QP, QC>())
    if (!e) e = setup_tv<DIM, QP, QC, 0, true>();
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

template <int DIM, int QP, int QC, int VAR, bool FAST = false>
int launch_tv(const DevParams& p, int stage, cudaStream_t s) {
  using C = TileCfg<DIM, VAR>;
  const dim3 grid((p.nx + C::TX - 1) / C::TX, DIM == 2 ? (p.ny + C::TY - 1) / C::TY : 1);
  switch (stage) {
    case kStage3:
      mixed_stage_kernel<DIM, QP, QC, kStage3, VAR, FAST>
          <<<grid, C::NT, smem_bytes<DIM, QP, QC, VAR, kStage3>(), s>>>(p);
      break;
    case kStage4:
      mixed_stage_kernel<DIM, QP, QC, kStage4, VAR, FAST>
          <<<grid, C::NT, smem_bytes<DIM, QP, QC, VAR, kStage4>(), s>>>(p);
      break;
    default:
      mixed_stage_kernel<DIM, QP, QC, kFinal, VAR, FAST>
          <<<grid, C::NT, smem_bytes<DIM, QP, QC, VAR, kFinal>(), s>>>(p);
      break;
  }
  return (int)cudaGetLastError();
}

template <int DIM, int QP, int QC>
int launch_prep(const DevParams& p, cudaStream_t s) {
  const int nt = 128;
  const int64_t nb = (p.N + nt - 1) / nt;
  mixed_prep_kernel<DIM, QP, QC><<<(unsigned)nb, nt, 0, s>>>(p);
  return (int)cudaGetLastError();
}

template <int DIM, int QP, int QC>
int launch_t(const DevParams& p, int stage, cudaStream_t s) {
  if (stage == kPrep) return launch_prep<DIM, QP, QC>(p, s);
  if constexpr (DIM == 1) {
    // 1-D problems pick their tile shape by length (single_1d_variant)
    switch (single_1d_variant(p.nx)) {
      case 1: return launch_tv<1, QP, QC, 1>(p, stage, s);
      case 3: return launch_tv<1, QP, QC, 3>(p, stage, s);
      case 4: return launch_tv<1, QP, QC, 4>(p, stage, s);
      default: return launch_tv<1, QP, QC, 0>(p, stage, s);
    }
  }
  if constexpr (fast_lattice<DIM, QP, QC>()) {
    // every tile full: the instance without the per-cell paths
    if (p.nx % TileCfg<2, 0>::TX == 0 && p.ny % TileCfg<2, 0>::TY == 0)
      return launch_tv<DIM, QP, QC, 0, true>(p, stage, s);
  }
  return launch_tv<DIM, QP, QC, 0>(p, stage, s);
}

template <int QP, int QC, int VAR>
int launch_batch_v(const DevParams& p, int stage, cudaStream_t s) {
  using C = TileCfg<1, VAR>;
  const int grid = p.bgrid > 0 ? p.bgrid : 1;
  switch (stage) {
    case kPrep: return launch_prep<1, QP, QC>(p, s);
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
    out[i] = (double)hi[i] + (double)lo[i];  // the pair's exact sum, rounded once
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
