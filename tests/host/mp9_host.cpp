// Host build of the device MP-9 routine (fdlb_mp9.cuh) for CPU unit tests:
// the CUDA qualifiers become plain inline functions and the bit casts go
// through memcpy.  Exposes mp9_face(v[9]) and mp9_march(line, n, sgn, out).
#include <cmath>
#include <cstring>
#define __device__
#define __forceinline__ inline
#define __restrict__
static inline long long __double_as_longlong(double x) { long long b; std::memcpy(&b, &x, 8); return b; }
static inline double __longlong_as_double(long long b) { double x; std::memcpy(&x, &b, 8); return x; }
using std::fma;
// binary32 intrinsics as the host's IEEE operations (built with -ffp-contract=off)
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
#include "../../paper_1909_08390_gb300/csrc/fdlb_mp9.cuh"

extern "C" double mp9_face(const double* v9) {
  // a one-interface march from the window v9 = F_{s-4..s+4}
  double out = 0.0;
  fdlb::mp9_march_fp64<1>(v9 + 4, 1, &out, 1);
  return out;
}

// interfaces 0..n of a line of n cells given with 5 ghosts per side
// (ext[0..n+9], cell c at ext[c+5]); out[i] = value at interface i (between
// cells i-1 and i) for velocity sign sgn, marched in segments of 8 or 1.
extern "C" void mp9_line(const double* ext, int n, int sgn, double* out) {
  for (int i = 0; i <= n; ++i) {
    const int up = (sgn > 0 ? i - 1 : i) + 5;
    fdlb::mp9_march_fp64<1>(ext + up, sgn, out + i, 1);
  }
}
extern "C" void mp9_line_march8(const double* ext, int n, int sgn, double* out) {
  // n + 1 must be a multiple of 8
  for (int i0 = 0; i0 <= n; i0 += 8) {
    const int first = sgn > 0 ? i0 : i0 + 7;
    const int up = (sgn > 0 ? first - 1 : first) + 5;
    fdlb::mp9_march_fp64<8>(ext + up, sgn, out + first, sgn);
  }
}

// bits of the device's one-operation DM = minmod4(4a - b, 4b - a, a, b)
extern "C" long long mp9_dm_bits(double a, double b) { return fdlb::dm_bits(a, b); }

// the binary32 interface value of the window v9 = F_{s-4..s+4}
extern "C" float mp9_face_f32(const float* v9) {
  float out = 0.0f;
  fdlb::mp9_march_fp32<1>(v9 + 4, 1, &out, 1);
  return out;
}
