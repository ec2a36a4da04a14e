// FP64 exponential for the rate evaluation, written from the table-driven method of
// P. T. P. Tang, "Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15 (1989):
//   x = (32 m + j) ln2/32 + r,  |r| <= ln2/64,   exp(x) = 2^m * 2^(j/32) * exp(r),
// with ln2/32 split in two parts (the first has 15 trailing zero bits so that
// N * L1 is exact for |N| < 2^15), exp(r) - 1 by its Taylor polynomial of degree 6
// (truncation below 3e-18 relative for |r| <= ln2/64), 2^(j/32) from a table of 32
// correctly rounded doubles, and 2^m applied to the exponent field with integer
// arithmetic.  Arguments outside |x| <= 700 (and NaN) take the library exp.
#pragma once
#include <cuda_runtime.h>

namespace mri {

constexpr double kExpInvL = 46.166241308446828;              // 32 / ln 2
constexpr double kExpL1 = 0x1.62e42fefa0000p-6;              // ln2/32, leading 38 bits
constexpr double kExpL2 = 0x1.cf79abc9e3b3ap-45;             // ln2/32 - L1
constexpr double kExpShift = 6755399441055744.0;             // 1.5 * 2^52: round to integer

__device__ __forceinline__ double exp_tab(double x, const double* __restrict__ tab32) {
  const int hx = __double2hiint(x) & 0x7fffffff;
  if (hx >= 0x4085E000) return exp(x);                      // |x| >= 700, Inf or NaN
  const double t = fma(x, kExpInvL, kExpShift);
  const int N = __double2loint(t);
  const double kd = t - kExpShift;
  double r = fma(-kd, kExpL1, x);
  r = fma(-kd, kExpL2, r);
  double p = fma(r, 1.0 / 720.0, 1.0 / 120.0);
  p = fma(p, r, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  p = p * r;                                                 // exp(r) - 1
  const double s = tab32[N & 31];
  const double v = fma(s, p, s);
  return __hiloint2double(__double2hiint(v) + (N >> 5) * 1048576, __double2loint(v));
}

}  // namespace mri
