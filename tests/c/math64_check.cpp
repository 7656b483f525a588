// Error bound of the float64 exp / expm1 pair used by the plain form, built
// for the host, and the exact float32 product it takes: both results of the
// pair against long-double expl / expm1l, in units of the last place of the
// float64 nearest the reference.  Exit status 0 when,
// for every y >= -708.3, e^y is within 0.6 ulp and e^y - 1 within 2 ulp,
// every y below -709.5 gives (0, -1) and the y between give one or the
// other, and every exact product equals the float64 product; prints the
// worst cases either way.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "vrc_math64.h"

static uint64_t state = 0x9e3779b97f4a7c15ull;
static double uniform01() {  // xorshift64* (Vigna 2016), 53-bit mantissa
  state ^= state >> 12;
  state ^= state << 25;
  state ^= state >> 27;
  return (double)((state * 0x2545f4914f6cdd1dull) >> 11) * 0x1.0p-53;
}

static double ulps(double got, long double ref) {
  const double r = (double)ref;
  if (r == 0.0) return got == 0.0 ? 0.0 : INFINITY;
  const double u = nextafter(fabs(r), INFINITY) - fabs(r);
  return (double)(fabsl((long double)got - ref) / (long double)u);
}

static double worst_ey = 0, worst_em = 0, at_ey = 0, at_em = 0;
static long n_checked = 0, n_bad_range = 0;

// yf: the float32 estimate of y that the kernels pass (y rounded to float32),
// or one float32 ulp either side of it.
static void check_one(double y, float yf) {
  double ey, em;
  vrc::m64::exp_expm1(y, yf, &ey, &em);
  const bool zero_pair = ey == 0.0 && em == -1.0;
  if (y < -709.5 || (y < -708.3 && zero_pair)) {
    if (!zero_pair && n_bad_range++ < 5) printf("below range y=%.17g: got (%.17g, %.17g)\n", y, ey, em);
    return;
  }
  const double e1 = ulps(ey, expl((long double)y));
  const double e2 = ulps(em, expm1l((long double)y));
  if (!(e1 <= worst_ey)) { worst_ey = e1; at_ey = y; }
  if (!(e2 <= worst_em)) { worst_em = e2; at_em = y; }
  ++n_checked;
}

static void check(double y) {
  const float f = (float)y;
  check_one(y, f);
  check_one(y, nextafterf(f, -INFINITY));
  check_one(y, nextafterf(f, INFINITY));
}

int main() {
  check(0.0);
  check(-0.0);
  for (int i = 0; i < 2000000; ++i) check(-760.0 * uniform01());       // whole range
  for (int i = 0; i < 1000000; ++i) check(-8.0 * uniform01());         // typical Sigma l
  for (int i = 0; i < 1000000; ++i) check(-pow(10.0, -300.0 + 302.0 * uniform01()));  // tiny to 100
  // either side of reduction boundaries (y = (n + 1/2) ln2/N) and of
  // n ln2/N: every n below 2^17, then every 7th down to the end of the range
  const double c = 0.6931471805599453 / vrc::m64::kTabSize;
  for (int n = 0; n < 1024 * 2050; n += (n < (1 << 17) ? 1 : 7)) {
    for (int d = -4; d <= 4; ++d) {
      check(-(n + 0.5) * c + d * 2e-16 * (1.0 + n * c));
      check(-n * c + d * 2e-16 * (1.0 + n * c));
    }
  }
  double ey, em;
  vrc::m64::exp_expm1(0.0, 0.0f, &ey, &em);
  const bool exact0 = ey == 1.0 && em == 0.0;
  vrc::m64::exp_expm1(-1e-300, -0.0f, &ey, &em);
  const bool tiny = ey == 1.0 && em == -1e-300;
  // reciprocal: normal float32 s from 2^-126 to 2^128 on a stride of 997 bit
  // patterns, against the long-double quotient and the float64 division
  long n_rcp = 0, rcp_off = 0;
  double worst_rcp = 0;
  for (uint32_t b = 0x00800000u; b <= 0x7f7fffffu; b += 997u) {
    float f;
    memcpy(&f, &b, sizeof f);
    const double got = vrc::m64::rcp(f), want = 1.0 / (double)f;
    const double u = ulps(got, 1.0L / (long double)f);
    if (u > worst_rcp) worst_rcp = u;
    rcp_off += got != want;
    ++n_rcp;
  }
  // exact product of two float32: bit for bit the float64 product, over
  // random normal pairs, zero and subnormal factors
  long prod_off = 0, n_prod = 0;
  for (int i = 0; i < 4000000; ++i) {
    const uint64_t u = (uint64_t)(uniform01() * 0x1p53);
    uint32_t ba = (uint32_t)u & 0x7fffffffu, bb = (uint32_t)(u >> 21) & 0x7fffffffu;
    if (i % 97 == 0) ba &= 0x007fffffu;  // subnormal or zero
    if (i % 89 == 0) bb = 0u;
    if ((ba >> 23) == 0xffu || (bb >> 23) == 0xffu) continue;
    float a, b;
    memcpy(&a, &ba, sizeof a);
    memcpy(&b, &bb, sizeof b);
    const double got = vrc::m64::exact_product(a, b), want = (double)a * (double)b;
    prod_off += memcmp(&got, &want, sizeof got) != 0;
    ++n_prod;
  }
  printf("exact product: %ld pairs, %ld differ from the float64 product\n", n_prod, prod_off);
  printf("rcp: %ld floats, worst %.3f ulp, %ld differ from the rounded quotient\n", n_rcp, worst_rcp,
         rcp_off);
  printf("checked %ld: worst exp %.3f ulp at y=%.17g, worst expm1 %.3f ulp at y=%.17g; "
         "below-range failures %ld; exact at 0: %d; tiny: %d\n",
         n_checked, worst_ey, at_ey, worst_em, at_em, n_bad_range, exact0, tiny);
  return (worst_ey <= 0.6 && worst_em <= 2.0 && n_bad_range == 0 && exact0 && tiny &&
          worst_rcp <= 0.51 && prod_off == 0) ? 0 : 1;
}
