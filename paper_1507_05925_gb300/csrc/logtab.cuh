// Natural logarithm in FP64 by table-driven argument reduction, for the output
// sums (one logarithm per source-target pair, on GB300's narrow FP64 pipe).
//
// Method: P. T. P. Tang, "Table-driven implementation of the logarithm
// function in IEEE floating-point arithmetic", ACM Trans. Math. Softw. 16(4),
// 1990.  Write x = 2^e m with m in [1, 2) and let j be the leading 7 bits of
// m's fraction, c_j = 1 + (j + 1/2)/128, so |m - c_j| <= 2^-8 and m - c_j is
// exact.  Then
//   log x = e log 2 + log c_j + log(1 + r),   r = (m - c_j)/c_j,  |r| < 2^-8,
// with log(1 + r) = r - r^2/2 + r^3/3 - ... + r^7/7 (the next term is below
// 2^-59 |r|).  The table holds (log c_j, 1/c_j) for j < 128; each block fills
// its own copy in shared memory (128 evaluations of the library logarithm and
// reciprocal), so nothing is kept between launches.  Arguments that are not
// positive normal finite numbers go to the library logarithm.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace bie {

constexpr int kLogTab = 128;

// Fill tab[0..127] (shared memory) with (log c_j, 1/c_j); call with at least
// 128 threads in the block, then synchronise before use.
__device__ __forceinline__ void log_table_fill(double2* tab) {
  const int j = threadIdx.x;
  if (j < kLogTab) {
    const double c = 1.0 + (j + 0.5) / kLogTab;
    tab[j] = make_double2(log(c), 1.0 / c);
  }
}

__device__ __forceinline__ double log_tab(double x, const double2* tab) {
  if (!(x >= 2.2250738585072014e-308) || !(x <= 1.7976931348623157e308)) return log(x);
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const int e = ((hi >> 20) & 0x7ff) - 1023;
  const int j = (hi >> 13) & 0x7f;
  const double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, lo);
  const double c = __hiloint2double(0x3ff00000 | (j << 13) | (1 << 12), 0);  // 1 + (j + 1/2)/128
  const double2 t = tab[j];
  const double r = (m - c) * t.y;
  // log(1 + r) = r + r^2 (-1/2 + r (1/3 + r (-1/4 + r (1/5 + r (-1/6 + r / 7)))))
  double p = fma(r, 1.0 / 7.0, -1.0 / 6.0);
  p = fma(p, r, 1.0 / 5.0);
  p = fma(p, r, -1.0 / 4.0);
  p = fma(p, r, 1.0 / 3.0);
  p = fma(p, r, -0.5);
  const double l1p = fma(p * r, r, r);
  return fma((double)e, 0.69314718055994530942, t.x + l1p);
}

}  // namespace bie
