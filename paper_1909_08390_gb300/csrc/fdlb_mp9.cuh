// fdlb_mp9.cuh -- MP-9 interface values with the Suresh-Huynh MP limiter
// (Sec. IV), evaluated along one line of a shared-memory tile.
//
// On GB300 the binary64 pipe issues two lanes per clock per SM, 64 times
// fewer than binary32, so the binary64 path spends that pipe on additions and
// multiplications only.  Every comparison, min/max, sign test, absolute
// value, power-of-two scaling and selection of the limiter runs on the
// integer pipe on the bit patterns: for IEEE doubles, k(x) = bits(x) ^
// ((bits(x) >> 63) & 0x7ff..f) is strictly increasing in x (with -0 ordered
// just below +0), so min/max/median of doubles are min/max/median of these
// int64 keys, and the key map is its own inverse.
//
// Formulation (all quantities are offsets from the upwind value F_s):
//   d_k  = F_{s+k+1} - F_{s+k}, k = -4..3        (forward differences)
//   a    = F^L - F_s = (-4 d_-4 + 37 d_-3 - 162 d_-2 + 479 d_-1 + 1120 d_0
//                       - 255 d_1 + 50 d_2 - 5 d_3) / 2520
//          (the printed 9-point stencil 4, -41, 199, -641, 1879, 1375, -305,
//          55, -5 over 2520, summed by parts)
//   C_j  = d_j - d_{j-1}                           (curvatures C_s, C_{s+-1})
//   DM+  = minmod4(4C_s - C_{s+1}, 4C_{s+1} - C_s, C_s, C_{s+1}), DM- likewise
//          with C_{s-1}; DM- of one interface is DM+ of the previous one
//   F^UL - F_s = 4 d_-1,  F^MD - F_s = (d_0 - DM+)/2,
//   F^LC - F_s = d_-1/2 + (4/3) DM-,  F_{s+1} - F_s = d_0
//   lo = max(min(0, d_0, md), min(0, ul, lc)), hi = min(max(0, d_0, md), max(0, ul, lc))
//   Fhat = F_s + clamp(a, lo, hi).
// The last line equals the paper's two cases: when (F^L - F_s)(F^L - F^MP) <=
// 0, a lies between 0 and minmod(d_0, 4 d_-1), an interval inside [lo, hi],
// so the clamp returns a; otherwise F^L + minmod(F^min - F^L, F^max - F^L) is
// F^L clamped to [F^min, F^max].  Evaluating it without the test keeps the
// warps of a line together (most lines of a developed flow have limited
// interfaces).  The bounds are formed at twice their value so that every
// halving becomes an exact power-of-two scaling.
#pragma once

#include <cstdint>

namespace fdlb {

// Bit casts.  On the device they are opaque register moves: a plain cast
// lets the compiler fold integer tests of the bits (a zero magnitude, an
// exponent range) back into binary64 compares, which run on the binary64
// pipe -- about five per interface, a third of the march's binary64 work.
#ifdef __CUDA_ARCH__
__device__ __forceinline__ long long dbits(double x) {
  long long r;
  asm("mov.b64 %0, %1;" : "=l"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double dfrom(long long b) {
  double r;
  asm("mov.b64 %0, %1;" : "=d"(r) : "l"(b));
  return r;
}
#else
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double dfrom(long long b) { return __longlong_as_double(b); }
#endif
constexpr long long kMag = 0x7fffffffffffffffLL;
constexpr long long kSign = (long long)0x8000000000000000ULL;

// order-preserving integer key (self-inverse)
__device__ __forceinline__ long long okey(long long b) { return b ^ ((b >> 63) & kMag); }
__device__ __forceinline__ long long kmin(long long a, long long b) { return a < b ? a : b; }
__device__ __forceinline__ long long kmax(long long a, long long b) { return a < b ? b : a; }

// Bits of DM = minmod4(4 ca - cb, 4 cb - ca, ca, cb) (the curvature bound of
// the MP limiter) with one binary64 operation.  DM is nonzero only if ca and
// cb share a sign; then, with m the one of smaller magnitude (ca on a tie)
// and M the other, 4 M - m has that sign and |4 M - m| >= 3 |M| >= |m|, so
// DM is 4 m - M if that also has the sign and |4 m - M| <= |m|, else m, and
// +0 when any of the four is zero or the signs differ.  On equal magnitudes
// the earlier argument is taken, as a sequential minmod4 does.
__device__ __forceinline__ long long dm_bits(double ca, double cb) {
  const long long ba = dbits(ca), bb = dbits(cb);
  const long long ma = ba & kMag, mb = bb & kMag;
  const bool a_small = ma <= mb;
  const double m = a_small ? ca : cb, M = a_small ? cb : ca;
  const long long bm = a_small ? ba : bb, mm = a_small ? ma : mb;
  const long long t = dbits(fma(4.0, m, -M));
  const long long mt = t & kMag;
  const bool nonzero = ((ba ^ bb) >= 0) && ((t ^ bm) >= 0) && (mm != 0) && (mt != 0);
  return nonzero ? (mt <= mm ? t : bm) : 0;
}

// bits of x * 2^K, K = 1..3, as an ordering key.  Exact for normal x with
// |x| < 2^(1024-K); zero stays zero; below the normal range the magnitude
// pattern is shifted (x * 2^K exactly while the result stays subnormal),
// above it saturates -- magnitudes that population differences of a valid
// state never take.
template <int K>
__device__ __forceinline__ long long key_times_pow2(long long b) {
  const long long m = b & kMag;
  const long long e = m >> 52;
  long long r;
  if (e == 0) r = m << K;
  else if (e > 2046 - K) r = 0x7fefffffffffffffLL;
  else r = m + ((long long)K << 52);
  return okey(r | (b & kSign));
}

struct Mp9Coef {
  // (-4, 37, -162, 479, 1120, -255, 50, -5) / 2520
  static constexpr double b0 = -4.0 / 2520.0, b1 = 37.0 / 2520.0, b2 = -162.0 / 2520.0,
                          b3 = 479.0 / 2520.0, b4 = 1120.0 / 2520.0, b5 = -255.0 / 2520.0,
                          b6 = 50.0 / 2520.0, b7 = -5.0 / 2520.0;
};

// Sliding state of one line: the upwind value F_s, the newest value, the
// eight differences d_-4..d_3, the curvatures C_{s-1}, C_s and DM- (the DM+
// of the previous interface).
struct Mp9Line {
  double fs[5];  // F_s .. F_{s+4}
  double d[8];   // d_-4 .. d_3
  double cm1, c0;
  long long dmm;
};

// Interface value for the current window; advances nothing.
__device__ __forceinline__ double mp9_face_fp64(const Mp9Line& L, double& c1_out,
                                                long long& dmp_out) {
  using B = Mp9Coef;
  const double* d = L.d;
  double a = B::b0 * d[0];
  a = fma(B::b1, d[1], a);
  a = fma(B::b2, d[2], a);
  a = fma(B::b3, d[3], a);
  a = fma(B::b4, d[4], a);
  a = fma(B::b5, d[5], a);
  a = fma(B::b6, d[6], a);
  a = fma(B::b7, d[7], a);
  const double c1 = d[5] - d[4];  // C_{s+1}
  const double c0 = L.c0;
  const long long dmp = dm_bits(c0, c1);
  // bounds at twice their value: 2 d_0, 2 md = d_0 - DM+, 2 ul = 8 d_-1,
  // 2 lc = d_-1 + (8/3) DM-, and 2a
  const long long k_d0 = key_times_pow2<1>(dbits(d[4]));
  const long long k_md = okey(dbits(d[4] - dfrom(dmp)));
  const long long k_ul = key_times_pow2<3>(dbits(d[3]));
  const long long k_lc = okey(dbits(fma(8.0 / 3.0, dfrom(L.dmm), d[3])));
  const long long k_a = key_times_pow2<1>(dbits(a));
  const long long lo = kmax(kmin(0, kmin(k_d0, k_md)), kmin(0, kmin(k_ul, k_lc)));
  const long long hi = kmin(kmax(0, kmax(k_d0, k_md)), kmax(0, kmax(k_ul, k_lc)));
  const double r2 = dfrom(okey(kmin(kmax(k_a, lo), hi)));
  c1_out = c1;
  dmp_out = dmp;
  return fma(0.5, r2, L.fs[0]);
}

// March NSTEP consecutive interfaces of one line.  `p` points at F_s (the
// upwind cell) of the first interface in march order, `ss` is the signed
// element stride from one interface's upwind cell to the next one's (upwind
// to downwind), `out` receives the interface values at out[t * ostep].
template <int NSTEP>
__device__ __forceinline__ void mp9_march_fp64(const double* __restrict__ p, int ss,
                                               double* __restrict__ out, int ostep) {
  Mp9Line L;
  double v[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) v[j] = p[(j - 4) * ss];
#pragma unroll
  for (int k = 0; k < 8; ++k) L.d[k] = v[k + 1] - v[k];
#pragma unroll
  for (int j = 0; j < 5; ++j) L.fs[j] = v[j + 4];
  L.cm1 = L.d[3] - L.d[2];
  L.c0 = L.d[4] - L.d[3];
  L.dmm = dm_bits(L.cm1, L.c0);
#pragma unroll
  for (int t = 0; t < NSTEP; ++t) {
    double c1;
    long long dmp;
    out[t * ostep] = mp9_face_fp64(L, c1, dmp);
    if (t + 1 < NSTEP) {
      const double vnew = p[(t + 5) * ss];
#pragma unroll
      for (int k = 0; k < 7; ++k) L.d[k] = L.d[k + 1];
      L.d[7] = vnew - L.fs[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) L.fs[j] = L.fs[j + 1];
      L.fs[4] = vnew;
      L.cm1 = L.c0;
      L.c0 = c1;
      L.dmm = dmp;
    }
  }
}

}  // namespace fdlb

namespace fdlb {

// binary32 version for the mixed-precision path: the same offset-form
// formulas on the binary32 pipe, with native min/max (cheap in binary32).
struct Mp9LineF {
  float fs[5];
  float d[8];
  float cm1, c0, dmm;
};

// Three-input minimum and maximum (one instruction on sm_100 and later).
__device__ __forceinline__ float fmin3f(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
#else
  return fminf(fminf(a, b), c);
#endif
}
__device__ __forceinline__ float fmax3f(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
#else
  return fmaxf(fmaxf(a, b), c);
#endif
}

// minmod4: the smallest of four positive values, the largest of four
// negative ones, else 0; that is max(min, 0) + min(max, 0).
__device__ __forceinline__ float minmod4f(float a, float b, float c, float d) {
  const float lo = fmin3f(a, b, fminf(c, d));
  const float hi = fmax3f(a, b, fmaxf(c, d));
  return fmaxf(lo, 0.0f) + fminf(hi, 0.0f);
}

// As in the binary64 face, the bounds and a are formed at twice their value
// (doubling the stencil's coefficients is exact), so that each bound takes
// one operation and the final halving is exact.  Returns the limited offset
// Fhat - F_s of the interface.
__device__ __forceinline__ float mp9_offset_fp32(const Mp9LineF& L, float& c1_out, float& dmp_out) {
  const float* d = L.d;
  float a2 = (2.0f * (-4.0f / 2520.0f)) * d[0];
  a2 = fmaf(2.0f * (37.0f / 2520.0f), d[1], a2);
  a2 = fmaf(2.0f * (-162.0f / 2520.0f), d[2], a2);
  a2 = fmaf(2.0f * (479.0f / 2520.0f), d[3], a2);
  a2 = fmaf(2.0f * (1120.0f / 2520.0f), d[4], a2);
  a2 = fmaf(2.0f * (-255.0f / 2520.0f), d[5], a2);
  a2 = fmaf(2.0f * (50.0f / 2520.0f), d[6], a2);
  a2 = fmaf(2.0f * (-5.0f / 2520.0f), d[7], a2);
  const float c1 = d[5] - d[4];
  const float c0 = L.c0;
  const float dmp = minmod4f(fmaf(4.0f, c0, -c1), fmaf(4.0f, c1, -c0), c0, c1);
  const float d0_2 = 2.0f * d[4];
  const float md2 = d[4] - dmp;
  const float ul2 = 8.0f * d[3];
  const float lc2 = fmaf(2.0f * (4.0f / 3.0f), L.dmm, d[3]);
  const float lo2 = fmaxf(fmin3f(0.0f, d0_2, md2), fmin3f(0.0f, ul2, lc2));
  const float hi2 = fminf(fmax3f(0.0f, d0_2, md2), fmax3f(0.0f, ul2, lc2));
  c1_out = c1;
  dmp_out = dmp;
  return 0.5f * fminf(fmaxf(a2, lo2), hi2);
}
__device__ __forceinline__ float mp9_face_fp32(const Mp9LineF& L, float& c1_out, float& dmp_out) {
  return __fadd_rn(mp9_offset_fp32(L, c1_out, dmp_out), L.fs[0]);
}

// March NSTEP consecutive interfaces of one whole line and write, for each of
// the NSTEP-1 cells between consecutive interfaces, its flux difference
// sgn (Fhat_right - Fhat_left) = d_-1 + a_cur - a_prev: the difference
// between the cell and its upwind neighbour plus the difference of the two
// interfaces' offsets a = Fhat - F_s from their upwind cells.  Formed from
// differences, it carries rounding relative to the variation along the line
// rather than to the values themselves.  out[t * ostep], t = 0..NSTEP-2, is
// the cell between interfaces t and t+1 in march order.
template <int NSTEP>
__device__ __forceinline__ void mp9_march_delta_fp32(const float* __restrict__ p, int ss,
                                                     float* __restrict__ out, int ostep) {
  Mp9LineF L;
  float v[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) v[j] = p[(j - 4) * ss];
#pragma unroll
  for (int k = 0; k < 8; ++k) L.d[k] = v[k + 1] - v[k];
#pragma unroll
  for (int j = 0; j < 5; ++j) L.fs[j] = v[j + 4];
  L.cm1 = L.d[3] - L.d[2];
  L.c0 = L.d[4] - L.d[3];
  L.dmm = minmod4f(fmaf(4.0f, L.c0, -L.cm1), fmaf(4.0f, L.cm1, -L.c0), L.c0, L.cm1);
  float aprev = 0.0f;
#pragma unroll
  for (int t = 0; t < NSTEP; ++t) {
    float c1, dmp;
    const float a = mp9_offset_fp32(L, c1, dmp);
    if (t > 0) out[(t - 1) * ostep] = __fsub_rn(__fadd_rn(L.d[3], a), aprev);
    aprev = a;
    if (t + 1 < NSTEP) {
      const float vnew = p[(t + 5) * ss];
#pragma unroll
      for (int k = 0; k < 7; ++k) L.d[k] = L.d[k + 1];
      L.d[7] = vnew - L.fs[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) L.fs[j] = L.fs[j + 1];
      L.fs[4] = vnew;
      L.cm1 = L.c0;
      L.c0 = c1;
      L.dmm = dmp;
    }
  }
}

template <int NSTEP>
__device__ __forceinline__ void mp9_march_fp32(const float* __restrict__ p, int ss,
                                               float* __restrict__ out, int ostep) {
  Mp9LineF L;
  float v[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) v[j] = p[(j - 4) * ss];
#pragma unroll
  for (int k = 0; k < 8; ++k) L.d[k] = v[k + 1] - v[k];
#pragma unroll
  for (int j = 0; j < 5; ++j) L.fs[j] = v[j + 4];
  L.cm1 = L.d[3] - L.d[2];
  L.c0 = L.d[4] - L.d[3];
  L.dmm = minmod4f(fmaf(4.0f, L.c0, -L.cm1), fmaf(4.0f, L.cm1, -L.c0), L.c0, L.cm1);
#pragma unroll
  for (int t = 0; t < NSTEP; ++t) {
    float c1, dmp;
    out[t * ostep] = mp9_face_fp32(L, c1, dmp);
    if (t + 1 < NSTEP) {
      const float vnew = p[(t + 5) * ss];
#pragma unroll
      for (int k = 0; k < 7; ++k) L.d[k] = L.d[k + 1];
      L.d[7] = vnew - L.fs[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) L.fs[j] = L.fs[j + 1];
      L.fs[4] = vnew;
      L.cm1 = L.c0;
      L.c0 = c1;
      L.dmm = dmp;
    }
  }
}

// Overloads so the stage kernel can march either storage type.
template <int NSTEP>
__device__ __forceinline__ void mp9_march(const double* p, int ss, double* out, int ostep) {
  mp9_march_fp64<NSTEP>(p, ss, out, ostep);
}
template <int NSTEP>
__device__ __forceinline__ void mp9_march(const float* p, int ss, float* out, int ostep) {
  mp9_march_fp32<NSTEP>(p, ss, out, ostep);
}

}  // namespace fdlb
