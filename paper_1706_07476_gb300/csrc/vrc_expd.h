// exp(y) and exp(y) - 1 in float64 for y <= 0, both from one argument
// reduction.  Used by the plain (float64) form of Eq. 4, where every segment
// needs the cell's transmitted factor e^-x and the path term's e^-x - 1.
//
// Method: Cody and Waite's additive range reduction (W. J. Cody and W. Waite,
// "Software Manual for the Elementary Functions", 1980): y = k ln2 + r with k
// the integer nearest y / ln2, so |r| <= ln2/2, and ln2 split into a float64
// head and a float64 tail so that y - k ln2_head is exact (|k| <= 1075 and the
// head's 53 bits leave the difference within 52 bits of 2^-2).  Then
//   e^r - 1 = q = r (1 + r/2! + r^2/3! + ... + r^12/13!)     (Taylor series)
// whose first omitted term, r^14/14!, is below 4.3e-18 for |r| <= 0.347, and
//   e^y     = 2^k (1 + q) = 2^k q + 2^k,
//   e^y - 1 = 2^k q + (2^k - 1),
// where 2^k - 1 is exact for -53 <= k <= 0 and both sums are free of
// cancellation (for k = 0 the second is q itself, which keeps full relative
// accuracy as y -> 0; for k <= -1 the magnitudes are at least 0.29).
//
// Range: y >= -708.3 keeps k >= -1022, so 2^k is a normal number built from
// its exponent bits.  Below that e^y < 2^-1021.9, and the pair returns
// (0, -1): every score that depends on it is below 1e-300.
// The host build of this header (no __CUDACC__) serves the CPU test that
// holds both results to a few ulp of a long-double reference.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define VRC_EXPD_FN __host__ __device__ __forceinline__
#else
#include <math.h>
#include <string.h>
#define VRC_EXPD_FN static inline
#endif

namespace vrc {
namespace expd {

VRC_EXPD_FN double bits_to_double(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
#endif
}

VRC_EXPD_FN uint32_t low_word(double d) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__double2loint(d);
#else
  uint64_t b;
  memcpy(&b, &d, sizeof b);
  return (uint32_t)b;
#endif
}

VRC_EXPD_FN double fmad(double a, double b, double c) {
#ifdef __CUDA_ARCH__
  return __fma_rn(a, b, c);
#else
  return fma(a, b, c);
#endif
}

// 1/ln2, and ln2 = kLn2Hi + kLn2Lo to about 2^-110 (both the float64 values
// nearest ln2 and nearest ln2 - kLn2Hi).
constexpr double kInvLn2 = 1.4426950408889634;
constexpr double kLn2Hi = 0x1.62e42fefa39efp-1;
constexpr double kLn2Lo = 0x1.abc9e3b39803fp-56;
// 1.5 * 2^52: adding it rounds to an integer held in the low mantissa bits.
constexpr double kRound = 6755399441055744.0;
// Below this y, k would leave the normal exponent range.
constexpr double kYMin = -708.3;

// Writes e^y to *ey and e^y - 1 to *em1, for y <= 0 (not NaN).
VRC_EXPD_FN void exp_expm1(double y, double *ey, double *em1) {
  const double t = fmad(y, kInvLn2, kRound);  // k + 1.5*2^52, k = nearest(y/ln2)
  const double kd = t - kRound;
  const uint32_t k = low_word(t);  // two's complement of k
  double r = fmad(-kd, kLn2Hi, y);  // exact
  r = fmad(-kd, kLn2Lo, r);
  // q = r * sum_{j=0}^{12} r^j / (j+1)!, coefficients 1/(j+1)! (Horner)
  double p = 1.6059043836821613e-10;  // 1/13!
  p = fmad(p, r, 2.08767569878681e-09);   // 1/12!
  p = fmad(p, r, 2.505210838544172e-08);  // 1/11!
  p = fmad(p, r, 2.755731922398589e-07);  // 1/10!
  p = fmad(p, r, 2.7557319223985893e-06); // 1/9!
  p = fmad(p, r, 2.48015873015873e-05);   // 1/8!
  p = fmad(p, r, 1.984126984126984e-04);  // 1/7!
  p = fmad(p, r, 1.388888888888889e-03);  // 1/6!
  p = fmad(p, r, 8.333333333333333e-03);  // 1/5!
  p = fmad(p, r, 4.1666666666666664e-02); // 1/4!
  p = fmad(p, r, 1.6666666666666666e-01); // 1/3!
  p = fmad(p, r, 0.5);                    // 1/2!
  p = fmad(p, r, 1.0);
  const double q = p * r;
  const double s = bits_to_double((uint64_t)(k + 1023u) << 52);  // 2^k
  const bool in_range = y >= kYMin;
  *ey = in_range ? fmad(s, q, s) : 0.0;
  *em1 = in_range ? fmad(s, q, s - 1.0) : -1.0;
}

}  // namespace expd
}  // namespace vrc
