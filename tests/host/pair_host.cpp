// Host build of the mixed-precision kernels' binary32-pair arithmetic and of
// their equilibrium factors (the code between the markers in
// csrc/fdlb_mixed.cu, extracted by the test and compiled with the stand-ins
// below for the CUDA intrinsics: every operation rounded once, as on the
// device).  Exposes the axis factors g_k = sum_l c_lk a_l(u, T) (Eq.
// gExpanded) for the tests.
#include <cmath>
#include <cstdint>

#define __device__
#define __forceinline__ inline

struct float2 {
  float x, y;
};
inline float2 make_float2(float a, float b) { return float2{a, b}; }
inline float __fadd_rn(float a, float b) { return a + b; }
inline float __fsub_rn(float a, float b) { return a - b; }
inline float __fmul_rn(float a, float b) { return a * b; }
inline float2 __fadd2_rn(float2 a, float2 b) { return {a.x + b.x, a.y + b.y}; }
inline float2 __fmul2_rn(float2 a, float2 b) { return {a.x * b.x, a.y * b.y}; }
inline float2 __ffma2_rn(float2 a, float2 b, float2 c) {
  return {std::fmaf(a.x, b.x, c.x), std::fmaf(a.y, b.y, c.y)};
}
inline float2 f2s(float a) { return {a, a}; }
inline float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2s(-1.0f), a); }
using std::fmaf;
constexpr int kMaxQ = 16;

namespace fdlb {
#include "_build/pair_extract.inc"

template <int Q>
static void run(const float* ch, const float* cl, float uh, float ul, float Th, float Tl,
                float sh, float sl, float* gh, float* gl) {
  DF g[Q];
  axis_g_df<Q>(ch, cl, DF{uh, ul}, DF{Th, Tl}, DF{sh, sl}, g);
  for (int k = 0; k < Q; ++k) {
    gh[k] = g[k].hi;
    gl[k] = g[k].lo;
  }
}
}  // namespace fdlb

extern "C" int host_axis_g_df(int Q, const float* ch, const float* cl, float uh, float ul,
                              float Th, float Tl, float sh, float sl, float* gh, float* gl) {
  switch (Q) {
    case 3: fdlb::run<3>(ch, cl, uh, ul, Th, Tl, sh, sl, gh, gl); return 0;
    case 5: fdlb::run<5>(ch, cl, uh, ul, Th, Tl, sh, sl, gh, gl); return 0;
    case 8: fdlb::run<8>(ch, cl, uh, ul, Th, Tl, sh, sl, gh, gl); return 0;
    default: return -1;
  }
}

// the pair product and sum on their own
extern "C" void host_df_mul(float ah, float al, float bh, float bl, float* rh, float* rl) {
  const fdlb::DF r = fdlb::df_mul(fdlb::DF{ah, al}, fdlb::DF{bh, bl});
  *rh = r.hi;
  *rl = r.lo;
}
extern "C" void host_df_add(float ah, float al, float bh, float bl, float* rh, float* rl) {
  const fdlb::DF r = fdlb::df_add(fdlb::DF{ah, al}, fdlb::DF{bh, bl});
  *rh = r.hi;
  *rl = r.lo;
}
