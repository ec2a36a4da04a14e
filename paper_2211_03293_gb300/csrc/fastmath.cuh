// FP64 exponential for the rate evaluation, written from the table-driven method of
// P. T. P. Tang, "Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15 (1989), with a table of 128 entries:
//   x = (128 m + j) ln2/128 + r,  |r| <= ln2/256,   exp(x) = 2^m * 2^(j/128) * exp(r),
// with ln2/128 split in two parts (the first has 36 significant bits, so that
// N * L1 is exact for |N| < 2^17), exp(r) - 1 by its Taylor polynomial of degree 5
// (truncation below 6e-19 relative for |r| <= ln2/256), 2^(j/128) from a table of
// 128 correctly rounded doubles, and 2^m applied to the exponent field with integer
// arithmetic.  Arguments outside |x| <= 700 (and NaN) take the library exp.  (The
// larger table buys one FP64 instruction per exponential over 32 entries.)
//
// FP64 natural logarithm, written from the table-driven method of P. T. P. Tang,
// "Table-driven implementation of the logarithm function in IEEE floating-point
// arithmetic", ACM TOMS 16 (1990):
//   x = 2^k m, m in [1, 2),  F = 1 + j/128 the nearest multiple of 1/128 to m,
//   log(x) = k ln2 + log(F) + log1p(u),  u = (m - F)/F,  |u| <= 2^-8,
// with m - F exact, 1/F from a table, log(F) and ln2 each split in a leading part
// with trailing zero bits (42 and 32 fractional bits, so k ln2_hi + log(F)_hi is
// exact) and a trailing part, and log1p(u) by its series to degree 8 (relative
// truncation below u^8/9 < 1e-20).  Zero, negative, subnormal, infinite and NaN
// arguments take the library log.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

namespace mri {

constexpr int kExpTab = 128;                                 // entries of the table 2^(j/128)
constexpr double kExpInvL = 184.66496523378731;              // 128 / ln 2
constexpr double kExpL1 = 0x1.62e42fefa0000p-8;              // ln2/128, leading 36 significant bits
constexpr double kExpL2 = 0x1.cf79abc9e3b3ap-47;             // ln2/128 - L1
constexpr double kExpShift = 6755399441055744.0;             // 1.5 * 2^52: round to integer

inline void fill_exp_table(double* t) {
  for (int j = 0; j < kExpTab; ++j) t[j] = (double)std::exp2l((long double)j / (long double)kExpTab);
}

__device__ __forceinline__ double exp_tab(double x, const double* __restrict__ tab) {
  const int hx = __double2hiint(x) & 0x7fffffff;
  if (hx >= 0x4085E000) return exp(x);                      // |x| >= 700, Inf or NaN
  const double t = fma(x, kExpInvL, kExpShift);
  const int N = __double2loint(t);
  const double kd = t - kExpShift;
  double r = fma(-kd, kExpL1, x);
  r = fma(-kd, kExpL2, r);
  double p = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  p = p * r;                                                 // exp(r) - 1
  const double s = tab[N & (kExpTab - 1)];
  const double v = fma(s, p, s);
  return __hiloint2double(__double2hiint(v) + (N >> 7) * 1048576, __double2loint(v));
}

// exp(x) and exp(-x) from one argument reduction (the method of exp_tab): with
// x = N ln2/128 + r, exp(x) = 2^(N>>7) 2^((N&127)/128) e^r and exp(-x) =
// 2^((-N)>>7) 2^(((-N)&127)/128) e^-r, and e^(+-r) - 1 = E(r) +- O(r) from the even
// and odd parts of the same degree-5 Taylor polynomial.  |x| >= 700 and NaN take
// the library exp.
__device__ __forceinline__ void exp_pair(double x, const double* __restrict__ tab, double& ep, double& em) {
  const int hx = __double2hiint(x) & 0x7fffffff;
  if (hx >= 0x4085E000) {
    ep = exp(x);
    em = exp(-x);
    return;
  }
  const double t = fma(x, kExpInvL, kExpShift);
  const int N = __double2loint(t);
  const double kd = t - kExpShift;
  double r = fma(-kd, kExpL1, x);
  r = fma(-kd, kExpL2, r);
  const double r2 = r * r;
  const double ev = r2 * fma(r2, 1.0 / 24.0, 0.5);                          // r^2/2 + r^4/24
  const double od = r * fma(fma(r2, 1.0 / 120.0, 1.0 / 6.0), r2, 1.0);     // r + r^3/6 + r^5/120
  const int Nm = -N;
  const double sp = tab[N & (kExpTab - 1)], sm = tab[Nm & (kExpTab - 1)];
  const double vp = fma(sp, ev + od, sp);
  const double vm = fma(sm, ev - od, sm);
  ep = __hiloint2double(__double2hiint(vp) + (N >> 7) * 1048576, __double2loint(vp));
  em = __hiloint2double(__double2hiint(vm) + (Nm >> 7) * 1048576, __double2loint(vm));
}

// table: [0, 129) 1/F, [129, 258) log(F) leading, [258, 387) log(F) trailing, then
// ln2 leading and trailing
constexpr int kLogTabDoubles = 389;

inline void fill_log_table(double* t) {
  for (int j = 0; j <= 128; ++j) {
    const long double F = 1.0L + (long double)j / 128.0L;
    const long double lg = logl(F);
    const double hi = std::ldexp(std::nearbyint(std::ldexp((double)lg, 42)), -42);
    t[j] = (double)(1.0L / F);
    t[129 + j] = hi;
    t[258 + j] = (double)(lg - (long double)hi);
  }
  const long double ln2 = logl(2.0L);
  const double hi = std::ldexp(std::floor(std::ldexp((double)ln2, 32)), -32);
  t[387] = hi;
  t[388] = (double)(ln2 - (long double)hi);
}

__device__ __forceinline__ double log_tab(double x, const double* __restrict__ t) {
  const long long b = __double_as_longlong(x);
  const int hx = (int)(b >> 32);
  if (hx < 0x00100000 || hx >= 0x7ff00000) return log(x);   // <= 0, subnormal, Inf, NaN
  const long long mant = b & 0x000fffffffffffffLL;
  const int j = (int)(((mant >> 44) + 1) >> 1);               // 0..128
  const double m = __longlong_as_double(mant | 0x3ff0000000000000LL);
  const double F = __longlong_as_double(0x3ff0000000000000LL + ((long long)j << 45));
  const double u = (m - F) * t[j];
  // log1p(u) = u + u^2 p(u)
  double p = fma(u, -1.0 / 8.0, 1.0 / 7.0);
  p = fma(p, u, -1.0 / 6.0);
  p = fma(p, u, 0.2);
  p = fma(p, u, -0.25);
  p = fma(p, u, 1.0 / 3.0);
  p = fma(p, u, -0.5);
  // k as a double through the 1.5 * 2^52 shift (k = biased exponent - 1023)
  const double kd = __longlong_as_double(0x4338000000000000LL + ((hx >> 20) - 1023)) - 6755399441055744.0;
  const double lo = fma(p, u * u, u + fma(kd, t[388], t[258 + j]));
  return fma(kd, t[387], t[129 + j]) + lo;
}

}  // namespace mri
