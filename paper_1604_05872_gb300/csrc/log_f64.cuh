// Natural logarithm in FP64 arithmetic for the Neo-Hookean ln det F.
//
// Table-driven (P. T. P. Tang, ACM TOMS 16(4), 1990): x = 2^k m with m in
// [1, 2); the seven leading fraction bits of m pick an interval j with centre
// c_j; with inv_j = RN(1 / c_j) and L_j = -ln inv_j (log_table.h),
//   ln x = k ln 2 + L_j + log1p(r),   r = m inv_j - 1 (one rounding, |r| < 2^-7),
// and log1p(r) is its Taylor polynomial to degree 8 (truncation below 2^-56
// relative).  Intervals from sqrt 2 up are shifted by ln 2 so that arguments near
// 1 from either side meet a small or zero L_j: no cancellation there.
//
// Cost: 13 FP64 operations, one 16-byte table load and integer bit handling
// (the exponent split, subnormal normalisation and k as a double are integer
// work: on this GPU the FP64 pipe runs about 2 lane-operations per SM per clock,
// 64 times slower than FP32).  Accuracy for finite x > 0, subnormals included:
// a few units in the last place.  Other arguments (zero, negative, inf, NaN)
// give unspecified values: callers test det F first.
#pragma once
#include <cstdint>

#include "log_table.h"

namespace fea {

__device__ __forceinline__ double log_f64(double x) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  int k = -1023;
  if ((b >> 52) == 0) {  // subnormal: normalise by an integer shift
    const int s = __clzll((long long)b) - 11;
    b <<= s;
    k -= s;
  }
  const uint32_t hi = (uint32_t)(b >> 32);
  const int j = (int)((hi >> 13) & 0x7fu);
  k += (int)(hi >> 20) + (j >= kLogSplit ? 1 : 0);
  const double m = __longlong_as_double((long long)((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
  const double2 t = __ldg(&kLogTab[j]);
  const double r = fma(m, t.x, -1.0);
  // log1p(r) = r + r^2 (-1/2 + r (1/3 + r (-1/4 + r (1/5 + r (-1/6 + r (1/7 - r / 8))))))
  double q = fma(-0.125, r, 1.0 / 7.0);
  q = fma(q, r, -1.0 / 6.0);
  q = fma(q, r, 0.2);
  q = fma(q, r, -0.25);
  q = fma(q, r, 1.0 / 3.0);
  q = fma(q, r, -0.5);
  const double p = fma(r * r, q, r);
  // k as a double without a conversion instruction: 2^52 + 2^31 + k, minus 2^52 + 2^31
  const double kd = __hiloint2double(0x43300000, (int)((uint32_t)k + 0x80000000u)) - 4503601774854144.0;
  return fma(kd, kLn2Hi, t.y) + fma(kd, kLn2Lo, p);
}

}  // namespace fea
