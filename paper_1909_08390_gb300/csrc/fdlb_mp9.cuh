// fdlb_mp9.cuh -- MP-9 interface values with the Suresh-Huynh MP limiter
// (Sec. IV), evaluated along one line of a shared-memory tile.
//
// On GB300 the binary64 pipe issues two lanes per clock per SM, 64 times
// fewer than binary32, so the binary64 path spends that pipe on additions and
// multiplications only.  Every comparison, min/max, sign test, absolute
// value and selection of the limiter runs on the integer pipe on the bit
// patterns: for IEEE doubles, k(x) = bits(x) ^ ((bits(x) >> 63) & 0x7ff..f)
// is strictly increasing in x (with -0 ordered just below +0), so
// min/max/median of doubles are min/max/median of these int64 keys, and the
// key map is its own inverse.
//
// The linear 9-point value is written on forward differences
// d_k = F_{s+k+1} - F_{s+k} (k = -4..3, s the upwind cell):
//   F^L - F_s = (-4 d_-4 + 37 d_-3 - 162 d_-2 + 479 d_-1 + 1120 d_0
//                - 255 d_1 + 50 d_2 - 5 d_3) / 2520,
// which is the printed stencil (coefficients 4, -41, 199, -641, 1879, 1375,
// -305, 55, -5 over 2520) summed by parts.  Marching along a line, each
// difference is computed once and slides through registers.
#pragma once

#include <cstdint>

namespace fdlb {

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double dfrom(long long b) { return __longlong_as_double(b); }
constexpr long long kMag = 0x7fffffffffffffffLL;

// order-preserving integer key (self-inverse)
__device__ __forceinline__ long long okey(long long b) { return b ^ ((b >> 63) & kMag); }
__device__ __forceinline__ long long kmin(long long a, long long b) { return a < b ? a : b; }
__device__ __forceinline__ long long kmax(long long a, long long b) { return a < b ? b : a; }

// four-argument minmod on bit patterns: if all four share a sign and none is
// zero, the one of smallest magnitude, else +0.
__device__ __forceinline__ long long minmod4_bits(long long a, long long b, long long c,
                                                  long long d) {
  const bool same = ((a ^ b) >= 0) && ((a ^ c) >= 0) && ((a ^ d) >= 0);
  const long long ma = a & kMag, mb = b & kMag, mc = c & kMag, md = d & kMag;
  const bool nz = (ma != 0) && (mb != 0) && (mc != 0) && (md != 0);
  long long r = a, mr = ma;
  if (mb < mr) { r = b; mr = mb; }
  if (mc < mr) { r = c; mr = mc; }
  if (md < mr) { r = d; }
  return (same && nz) ? r : 0;
}

// |4x| as a magnitude bit pattern (x = +-0 gives 0).  Exact for normal x with
// |x| < 2^1021; below the normal range the pattern is shifted (4x exactly
// while |x| < 2^-1073), above it saturates -- magnitudes populations of a
// valid state never take.
__device__ __forceinline__ long long mag_times4(long long b) {
  const long long m = b & kMag;
  const long long e = m >> 52;
  if (e == 0) return m << 2;
  if (e > 2044) return 0x7fefffffffffffffLL;
  return m + (2LL << 52);
}

struct Mp9Coef {
  // (-4, 37, -162, 479, 1120, -255, 50, -5) / 2520
  static constexpr double b0 = -4.0 / 2520.0, b1 = 37.0 / 2520.0, b2 = -162.0 / 2520.0,
                          b3 = 479.0 / 2520.0, b4 = 1120.0 / 2520.0, b5 = -255.0 / 2520.0,
                          b6 = 50.0 / 2520.0, b7 = -5.0 / 2520.0;
};

// Interface value from the window v[0..8] = F_{s-4..s+4} (upwind
// orientation) and its differences d[0..7] = F_{s-3..s+4} - F_{s-4..s+3}.
__device__ __forceinline__ double mp9_face_fp64(const double (&v)[9], const double (&d)[8]) {
  using B = Mp9Coef;
  double a = B::b0 * d[0];
  a = fma(B::b1, d[1], a);
  a = fma(B::b2, d[2], a);
  a = fma(B::b3, d[3], a);
  a = fma(B::b4, d[4], a);
  a = fma(B::b5, d[5], a);
  a = fma(B::b6, d[6], a);
  a = fma(B::b7, d[7], a);
  const double Fs = v[4];
  const double FL = Fs + a;
  // (F^L - F_s)(F^L - F^MP) <= 0 with F^MP = F_s + minmod(d_0, 4 d_-1), i.e.
  // a lies between 0 and minmod(d_0, 4 d_-1) (both inclusive): keep F^L.
  const long long ba = dbits(a), b0 = dbits(d[4]), bm = dbits(d[3]);
  const long long ma = ba & kMag, m0 = b0 & kMag, mm = bm & kMag;
  const bool keep = (ma == 0) || (((b0 ^ bm) >= 0) && (m0 != 0) && (mm != 0) &&
                                  ((ba ^ b0) >= 0) && (ma <= m0) && (ma <= mag_times4(bm)));
  if (keep) return FL;
  // limited branch: curvatures, bounds, and the median
  const double Cm1 = d[3] - d[2];  // C_{s-1} = F_s - 2F_{s-1} + F_{s-2}
  const double C0 = d[4] - d[3];   // C_s
  const double Cp1 = d[5] - d[4];  // C_{s+1}
  const long long dmp = minmod4_bits(dbits(fma(4.0, C0, -Cp1)), dbits(fma(4.0, Cp1, -C0)),
                                     dbits(C0), dbits(Cp1));
  const long long dmm = minmod4_bits(dbits(fma(4.0, C0, -Cm1)), dbits(fma(4.0, Cm1, -C0)),
                                     dbits(C0), dbits(Cm1));
  const double FUL = fma(4.0, d[3], Fs);                          // F_s + 4 (F_s - F_{s-1})
  const double FMD = fma(0.5, d[4] - dfrom(dmp), Fs);             // (F_s + F_{s+1} - DM+)/2
  const double FLC = fma(4.0 / 3.0, dfrom(dmm), fma(0.5, d[3], Fs));
  const long long kFs = okey(dbits(Fs)), kFp1 = okey(dbits(v[5])), kMD = okey(dbits(FMD));
  const long long kUL = okey(dbits(FUL)), kLC = okey(dbits(FLC));
  const long long kmin1 = kmin(kFs, kmin(kFp1, kMD)), kmin2 = kmin(kFs, kmin(kUL, kLC));
  const long long kmax1 = kmax(kFs, kmax(kFp1, kMD)), kmax2 = kmax(kFs, kmax(kUL, kLC));
  const long long klo = kmax(kmin1, kmin2), khi = kmin(kmax1, kmax2);  // klo <= k(F_s) <= khi
  // F^L + minmod(F^min - F^L, F^max - F^L) = F^L clamped to [F^min, F^max]
  const long long kFL = okey(dbits(FL));
  return dfrom(okey(kmin(kmax(kFL, klo), khi)));
}

// March NSTEP consecutive interfaces of one line.  `p` points at v_0 (the
// upwind cell) of the first interface in march order, `ss` is the signed
// element stride from one interface's upwind cell to the next one's (upwind
// to downwind), `out` receives the interface values at out[t * ostep].
template <int NSTEP>
__device__ __forceinline__ void mp9_march_fp64(const double* __restrict__ p, int ss,
                                               double* __restrict__ out, int ostep) {
  double v[9], d[8];
#pragma unroll
  for (int j = 0; j < 9; ++j) v[j] = p[(j - 4) * ss];
#pragma unroll
  for (int k = 0; k < 8; ++k) d[k] = v[k + 1] - v[k];
#pragma unroll
  for (int t = 0; t < NSTEP; ++t) {
    out[t * ostep] = mp9_face_fp64(v, d);
    if (t + 1 < NSTEP) {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = v[j + 1];
      v[8] = p[(t + 5) * ss];
#pragma unroll
      for (int k = 0; k < 7; ++k) d[k] = d[k + 1];
      d[7] = v[8] - v[7];
    }
  }
}

}  // namespace fdlb
