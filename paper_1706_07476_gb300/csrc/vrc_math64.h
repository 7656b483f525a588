// Float64 helpers of the plain form: exp(y) and exp(y) - 1 for y <= 0 from
// one argument reduction, and 1/s for a float32 s.
//
// exp(y) and exp(y) - 1 in float64 for y <= 0, both from one argument
// reduction.  Used by the plain (float64) form of Eq. 4, where every segment
// needs the cell's transmitted factor e^-x and the path term's e^-x - 1.
//
// Method: Tang's table-driven reduction (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989) with Cody and Waite's two-part constant
// (W. J. Cody and W. Waite, "Software Manual for the Elementary Functions",
// 1980):
//   y = (64 m + j) ln2/64 + r,  n = 64 m + j an integer near 64 y / ln2,
//   e^y = 2^m 2^(j/64) e^r.
// n comes from a float32 estimate of y (relative error <= 2^-23, so n is
// the nearest integer or one off it near a half-integer): |r| <= 0.00555.
// ln2/64 is split into kC1 + kC2; y - n kC1 is exact in one fused
// multiply-add (the difference is below 2^-7 and spans at most 53 bits).
// e^r - 1 = q = r (1 + r/2! + r^2/3! + r^3/4! + r^4/5! + r^5/6!) (Taylor
// series; the first omitted term, r^6/7!, is below 6e-18 of |r|).  With
// 2^(j/64) = T_hi + T_lo (float64 head and tail, kExp2Tab) and s = 2^m:
//   c       = T_hi q + T_lo              (= 2^(j/64)(1 + q) - T_hi)
//   e^y     = s c + s T_hi
//   e^y - 1 = s c + (s T_hi - 1)
// s T_hi is exact, and s T_hi - 1 is exact for n >= -64 (s T_hi in [1/2, 1],
// Sterbenz) and rounded once otherwise, where |e^y - 1| >= 0.49; for n = 0
// the second line is q itself, which keeps full relative accuracy as y -> 0.
//
// Range: n >= -65408 keeps m >= -1022, so 2^m is a normal number built from
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
#define VRC_M64_FN __host__ __device__ __forceinline__
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

// 64/ln2 (float32), and ln2/64 = kC1 + kC2 to about 2^-115.
constexpr float kInvCf = 92.332482616893658f;
constexpr double kC1 = 0x1.62e42fefa39efp-7;
constexpr double kC2 = 0x1.abc9e3b39803fp-62;
// 1.5 * 2^23 and 1.5 * 2^52: adding one rounds to an integer held in the low
// mantissa bits (float32 for |n| < 2^22, float64 for |n| < 2^51).
constexpr float kRoundF = 12582912.0f;
constexpr double kRound = 6755399441055744.0;
constexpr uint32_t kRoundFBits = 0x4b400000u;
constexpr uint64_t kRoundBits = 0x4338000000000000ull;
// Smallest n with m = floor(n/64) >= -1022.
constexpr int32_t kNMin = -65408;

// 2^(j/64), j = 0..63: the nearest float64, and the nearest float64 to the
// remainder.
#ifdef __CUDACC__
__device__
#endif
static const double kExp2Tab[64][2] = {
    {0x1.0000000000000p+0, 0x0p+0},
    {0x1.02c9a3e778061p+0, -0x1.19083535b085dp-56},
    {0x1.059b0d3158574p+0, 0x1.d73e2a475b465p-55},
    {0x1.0874518759bc8p+0, 0x1.186be4bb284ffp-57},
    {0x1.0b5586cf9890fp+0, 0x1.8a62e4adc610bp-54},
    {0x1.0e3ec32d3d1a2p+0, 0x1.03a1727c57b53p-59},
    {0x1.11301d0125b51p+0, -0x1.6c51039449b3ap-54},
    {0x1.1429aaea92de0p+0, -0x1.32fbf9af1369ep-54},
    {0x1.172b83c7d517bp+0, -0x1.19041b9d78a76p-55},
    {0x1.1a35beb6fcb75p+0, 0x1.e5b4c7b4968e4p-55},
    {0x1.1d4873168b9aap+0, 0x1.e016e00a2643cp-54},
    {0x1.2063b88628cd6p+0, 0x1.dc775814a8495p-55},
    {0x1.2387a6e756238p+0, 0x1.9b07eb6c70573p-54},
    {0x1.26b4565e27cddp+0, 0x1.2bd339940e9d9p-55},
    {0x1.29e9df51fdee1p+0, 0x1.612e8afad1255p-55},
    {0x1.2d285a6e4030bp+0, 0x1.0024754db41d5p-54},
    {0x1.306fe0a31b715p+0, 0x1.6f46ad23182e4p-55},
    {0x1.33c08b26416ffp+0, 0x1.32721843659a6p-54},
    {0x1.371a7373aa9cbp+0, -0x1.63aeabf42eae2p-54},
    {0x1.3a7db34e59ff7p+0, -0x1.5e436d661f5e3p-56},
    {0x1.3dea64c123422p+0, 0x1.ada0911f09ebcp-55},
    {0x1.4160a21f72e2ap+0, -0x1.ef3691c309278p-58},
    {0x1.44e086061892dp+0, 0x1.89b7a04ef80d0p-59},
    {0x1.486a2b5c13cd0p+0, 0x1.3c1a3b69062f0p-56},
    {0x1.4bfdad5362a27p+0, 0x1.d4397afec42e2p-56},
    {0x1.4f9b2769d2ca7p+0, -0x1.4b309d25957e3p-54},
    {0x1.5342b569d4f82p+0, -0x1.07abe1db13cadp-55},
    {0x1.56f4736b527dap+0, 0x1.9bb2c011d93adp-54},
    {0x1.5ab07dd485429p+0, 0x1.6324c054647adp-54},
    {0x1.5e76f15ad2148p+0, 0x1.ba6f93080e65ep-54},
    {0x1.6247eb03a5585p+0, -0x1.383c17e40b497p-54},
    {0x1.6623882552225p+0, -0x1.bb60987591c34p-54},
    {0x1.6a09e667f3bcdp+0, -0x1.bdd3413b26456p-54},
    {0x1.6dfb23c651a2fp+0, -0x1.bbe3a683c88abp-57},
    {0x1.71f75e8ec5f74p+0, -0x1.16e4786887a99p-55},
    {0x1.75feb564267c9p+0, -0x1.0245957316dd3p-54},
    {0x1.7a11473eb0187p+0, -0x1.41577ee04992fp-55},
    {0x1.7e2f336cf4e62p+0, 0x1.05d02ba15797ep-56},
    {0x1.82589994cce13p+0, -0x1.d4c1dd41532d8p-54},
    {0x1.868d99b4492edp+0, -0x1.fc6f89bd4f6bap-54},
    {0x1.8ace5422aa0dbp+0, 0x1.6e9f156864b27p-54},
    {0x1.8f1ae99157736p+0, 0x1.5cc13a2e3976cp-55},
    {0x1.93737b0cdc5e5p+0, -0x1.75fc781b57ebcp-57},
    {0x1.97d829fde4e50p+0, -0x1.d185b7c1b85d1p-54},
    {0x1.9c49182a3f090p+0, 0x1.c7c46b071f2bep-56},
    {0x1.a0c667b5de565p+0, -0x1.359495d1cd533p-54},
    {0x1.a5503b23e255dp+0, -0x1.d2f6edb8d41e1p-54},
    {0x1.a9e6b5579fdbfp+0, 0x1.0fac90ef7fd31p-54},
    {0x1.ae89f995ad3adp+0, 0x1.7a1cd345dcc81p-54},
    {0x1.b33a2b84f15fbp+0, -0x1.2805e3084d708p-57},
    {0x1.b7f76f2fb5e47p+0, -0x1.5584f7e54ac3bp-56},
    {0x1.bcc1e904bc1d2p+0, 0x1.23dd07a2d9e84p-55},
    {0x1.c199bdd85529cp+0, 0x1.11065895048ddp-55},
    {0x1.c67f12e57d14bp+0, 0x1.2884dff483cadp-54},
    {0x1.cb720dcef9069p+0, 0x1.503cbd1e949dbp-56},
    {0x1.d072d4a07897cp+0, -0x1.cbc3743797a9cp-54},
    {0x1.d5818dcfba487p+0, 0x1.2ed02d75b3707p-55},
    {0x1.da9e603db3285p+0, 0x1.c2300696db532p-54},
    {0x1.dfc97337b9b5fp+0, -0x1.1a5cd4f184b5cp-54},
    {0x1.e502ee78b3ff6p+0, 0x1.39e8980a9cc8fp-55},
    {0x1.ea4afa2a490dap+0, -0x1.e9c23179c2893p-54},
    {0x1.efa1bee615a27p+0, 0x1.dc7f486a4b6b0p-54},
    {0x1.f50765b6e4540p+0, 0x1.9d3e12dd8a18bp-54},
    {0x1.fa7c1819e90d8p+0, 0x1.74853f3a5931ep-55},
};

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

// Writes e^y to *ey and e^y - 1 to *em1, for y <= 0 (not NaN); yf is y
// rounded to float32 (or any float32 within 2^-23 |y| of it).
VRC_M64_FN void exp_expm1(double y, float yf, double *ey, double *em1) {
  yf = yf > -1000.f ? yf : -1000.f;
  const float tf = fmaf_rn(yf, kInvCf, kRoundF);
  const int32_t n = (int32_t)(float_bits(tf) - kRoundFBits);  // nearest(64 yf / ln2)
  const double nd = bits_to_double(kRoundBits + (uint64_t)(int64_t)n) - kRound;
  double r = fmad(-nd, kC1, y);  // exact
  r = fmad(-nd, kC2, r);
  double p = 1.388888888888889e-03;       // 1/6!
  p = fmad(p, r, 8.333333333333333e-03);  // 1/5!
  p = fmad(p, r, 4.1666666666666664e-02); // 1/4!
  p = fmad(p, r, 1.6666666666666666e-01); // 1/3!
  p = fmad(p, r, 0.5);                    // 1/2!
  p = fmad(p, r, 1.0);
  const double q = p * r;  // e^r - 1
  double thi, tlo;
  table_entry((uint32_t)n & 63u, &thi, &tlo);
  const uint32_t m = (uint32_t)(n >> 6);  // floor(n / 64), two's complement
  const double s = bits_to_double((uint64_t)(m + 1023u) << 52);  // 2^m
  const double c = fmad(thi, q, tlo);
  const double a = s * thi;  // exact
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
