// Float64 helpers of the plain form: exp(y) and exp(y) - 1 for y <= 0 from
// one argument reduction, the exact product of two float32, and 1/s for a
// float32 s.
//
// exp(y) and exp(y) - 1 in float64 for y <= 0, both from one argument
// reduction.  Used by the plain (float64) form of Eq. 4, where every segment
// needs the cell's transmitted factor e^-x and the path term's e^-x - 1.
//
// Method: Tang's table-driven reduction (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989) with Cody and Waite's two-part constant
// (W. J. Cody and W. Waite, "Software Manual for the Elementary Functions",
// 1980), with N = 2048 table entries:
//   y = (N m + j) ln2/N + r,  n = N m + j an integer near N y / ln2,
//   e^y = 2^m 2^(j/N) e^r.
// n comes from a float32 estimate of y (relative error <= 2^-23, so n is
// within one of the nearest integer; |r| <= 0.00017 for |y| < 100 and
// <= 0.00034 everywhere).  ln2/N is split into kC1 + kC2 (kC1 the nearest
// float64); y - n kC1 is exact in one fused multiply-add: for n != 0 the
// difference is below 2^-11 and its lowest bit is no lower than y's or
// kC1's (2^-65 at the smallest |y| with n != 0, where |r| < 2^-12).
// e^r - 1 = q = r (1 + r/2! + r^2/3! + r^3/4!) (Taylor series; the first
// omitted term, r^4/5! of |r|, is below 1e-17 of |r| for |r| <= 0.00017 and
// below 2e-16 of |r| at 0.00034, where only e^y, to which it adds 1e-20,
// needs it).  With 2^(j/N) = T_hi + T_lo (float64 head and tail, kExp2Tab)
// and s = 2^m:
//   c       = T_hi q + T_lo              (= 2^(j/N)(1 + q) - T_hi)
//   e^y     = s c + s T_hi
//   e^y - 1 = s c + (s T_hi - 1)
// s T_hi is exact, and s T_hi - 1 is exact for n >= -N (s T_hi in [1/2,
// 1], Sterbenz) and rounded once otherwise, where |e^y - 1| >= 0.49; for
// n = 0 the second line is q itself, which keeps full relative accuracy as
// y -> 0.  A 2048-entry table (32 KiB) rather than 256 entries saves one
// series term.  n as a float64 and the exact product 2^m T_hi are built from
// integer fields, not with float64 arithmetic: 12 float64 operations here.
//
// Range: n >= kNMin keeps m >= -1022, so 2^m is a normal number built from
// its exponent bits (y >= -708.3 always qualifies).  Below it e^y < 2^-1021,
// and the pair returns (0, -1): every score that depends on it is below
// 1e-300.  The float32 estimate is clamped at -1000 before n is formed.
//
// kExp2Tab is written by vrc_math64_table.py (exact decimal arithmetic).  The
// host build of this header (no __CUDACC__) serves the CPU test that holds
// both results to 2 ulp of a long-double reference.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define VRC_M64_FN __device__ __forceinline__
#else
#include <math.h>
#include <string.h>
#define VRC_M64_FN static inline
#endif

namespace vrc {
namespace m64 {

VRC_M64_FN double bits_to_double(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
#endif
}

VRC_M64_FN uint64_t double_bits(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t b;
  memcpy(&b, &d, sizeof b);
  return b;
#endif
}

VRC_M64_FN uint32_t float_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t b;
  memcpy(&b, &f, sizeof b);
  return b;
#endif
}

VRC_M64_FN double fmad(double a, double b, double c) {
#ifdef __CUDA_ARCH__
  return __fma_rn(a, b, c);
#else
  return fma(a, b, c);
#endif
}

VRC_M64_FN float fmaf_rn(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}

// Table entries N = 2^kTabBits; N/ln2 (float32), and ln2/N = kC1 + kC2 to
// about 2^-120.
constexpr int kTabBits = 11;
constexpr int kTabSize = 1 << kTabBits;
constexpr float kInvCf = 2954.639443740597f;
constexpr double kC1 = 0x1.62e42fefa39efp-12;
constexpr double kC2 = 0x1.abc9e3b39803fp-67;
// 1.5 * 2^23: adding it rounds a float32 to an integer held in the low
// mantissa bits (for |n| < 2^22).
constexpr float kRoundF = 12582912.0f;
constexpr uint32_t kRoundFBits = 0x4b400000u;
// Smallest n with m = floor(n/N) >= -1022.
constexpr int32_t kNMin = -1022 * kTabSize;

#include "vrc_exp2_table.h"  // kExp2Tab[kTabSize][2]

VRC_M64_FN void table_entry(uint32_t j, double *hi, double *lo) {
#ifdef __CUDA_ARCH__
  const double2 v = __ldg(reinterpret_cast<const double2 *>(kExp2Tab[j]));
  *hi = v.x;
  *lo = v.y;
#else
  *hi = kExp2Tab[j][0];
  *lo = kExp2Tab[j][1];
#endif
}

// The float64 equal to an integer-valued float32 f (|f| < 2^24), built from
// f's sign, exponent (rebiased by 1023 - 127) and mantissa with integer
// operations; 0 maps to +0.
VRC_M64_FN double int_float_to_double(float f) {
  const uint32_t b = float_bits(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  return bits_to_double(((uint64_t)((b & 0x80000000u) | ((e + 896u) << 20) | ((b >> 3) & 0xfffffu)) << 32) |
                        ((uint64_t)(b << 29)));
}

// The float64 product of two float32 a, b >= 0, exact (two 24-bit
// significands give at most 48 bits), formed with integer operations: the
// significands' integer product (in [2^46, 2^48)) shifted into the float64
// fraction, and the sum of the exponents.  A zero factor gives +0;
// subnormal, infinite, NaN or negative inputs take the float64 multiply.
VRC_M64_FN double exact_product(float a, float b) {
  const uint32_t ba = float_bits(a), bb = float_bits(b);
  const uint32_t ea = ba >> 23, eb = bb >> 23;
  if (ea - 1u >= 254u || eb - 1u >= 254u) {
    if (ba == 0u || bb == 0u) return 0.0;
    return (double)a * (double)b;
  }
  const uint64_t P = (uint64_t)((ba & 0x7fffffu) | 0x800000u) * (uint64_t)((bb & 0x7fffffu) | 0x800000u);
  const uint32_t top = (uint32_t)(P >> 47);  // P in [2^(46+top), 2^(47+top))
  const uint64_t frac = (P << (6u - top)) & 0xfffffffffffffull;
  return bits_to_double(((uint64_t)(ea + eb + 769u + top) << 52) | frac);
}

// Writes e^y to *ey and e^y - 1 to *em1, for y <= 0 (not NaN); yf is y
// rounded to float32 (or any float32 within 2^-23 |y| of it).  The integer n
// (as a float64) and 2^m T_hi are formed with integer operations, which
// leaves 12 float64 operations here.
VRC_M64_FN void exp_expm1(double y, float yf, double *ey, double *em1) {
  yf = yf > -1000.f ? yf : -1000.f;
  const float tf = fmaf_rn(yf, kInvCf, kRoundF);
  const int32_t n = (int32_t)(float_bits(tf) - kRoundFBits);  // nearest(N yf / ln2)
  const double nd = int_float_to_double(tf - kRoundF);         // n, exactly (|n| < 2^22)
  double r = fmad(-nd, kC1, y);  // exact
  r = fmad(-nd, kC2, r);
  double p = 4.1666666666666664e-02;      // 1/4!
  p = fmad(p, r, 1.6666666666666666e-01); // 1/3!
  p = fmad(p, r, 0.5);                    // 1/2!
  p = fmad(p, r, 1.0);
  const double q = p * r;  // e^r - 1
  double thi, tlo;
  table_entry((uint32_t)n & (uint32_t)(kTabSize - 1), &thi, &tlo);
  const uint32_t m = (uint32_t)(n >> kTabBits);  // floor(n / N), two's complement
  const double s = bits_to_double((uint64_t)(m + 1023u) << 52);  // 2^m
  const double c = fmad(thi, q, tlo);
  // a = 2^m T_hi (exact): T_hi in [1, 2), so m goes into its exponent field
  // (m >= -1022 in range keeps a normal; out of range a is not used)
  const double a = bits_to_double(double_bits(thi) + ((uint64_t)(int64_t)(int32_t)m << 52));
  const bool in_range = n >= kNMin;
  *ey = in_range ? fmad(s, c, a) : 0.0;
  *em1 = in_range ? fmad(s, c, a - 1.0) : -1.0;
}

// 1/s in float64 for a float32 s > 0, from the float32 reciprocal r0 =
// 1/s (1 + d), |d| <= 2^-24 (correctly rounded), and one Newton-Raphson step
// taken to third order: with e = 1 - s r0 = -d (exact: s r0 is a 48-bit
// product), 1/s = r0 (1 + e + e^2 + ...), so r = r0 + r0 (e + e^2) has
// relative error d^3 <= 2^-72 before its final rounding (within 0.51 ulp).
// Three float64 operations in place of a division.  Inputs outside
// [2^-125, 2^125] (whose float32 reciprocal would overflow or lose bits to
// the subnormal range), infinities and NaN take the division.
VRC_M64_FN double rcp(float s) {
  if (!(s >= 0x1p-125f && s <= 0x1p125f)) return 1.0 / (double)s;
#ifdef __CUDA_ARCH__
  const float r0f = __frcp_rn(s);
#else
  const float r0f = 1.0f / s;
#endif
  const double sd = (double)s, r0 = (double)r0f;
  const double e = fmad(-sd, r0, 1.0);
  return fmad(r0, fmad(e, e, e), r0);
}

}  // namespace m64
}  // namespace vrc
