// Error bound of the float64 exp / expm1 pair used by the plain form, built
// for the host: both results against long-double expl / expm1l, in units of
// the last place of the float64 nearest the reference.  Exit status 0 when
// every in-range y (e^y normal) is within 2 ulp and every y below the range
// gives (0, -1); prints the worst cases either way.
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include "vrc_expd.h"

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

static void check(double y) {
  double ey, em;
  vrc::expd::exp_expm1(y, &ey, &em);
  if (y < vrc::expd::kYMin) {
    if (!(ey == 0.0 && em == -1.0)) {
      if (n_bad_range++ < 5) printf("below range y=%.17g: got (%.17g, %.17g)\n", y, ey, em);
    }
    return;
  }
  const double e1 = ulps(ey, expl((long double)y));
  const double e2 = ulps(em, expm1l((long double)y));
  if (!(e1 <= worst_ey)) { worst_ey = e1; at_ey = y; }
  if (!(e2 <= worst_em)) { worst_em = e2; at_em = y; }
  ++n_checked;
}

int main() {
  check(0.0);
  check(-0.0);
  for (int i = 0; i < 2000000; ++i) check(-760.0 * uniform01());       // whole range
  for (int i = 0; i < 1000000; ++i) check(-8.0 * uniform01());         // typical Sigma l
  for (int i = 0; i < 1000000; ++i) check(-pow(10.0, -300.0 + 302.0 * uniform01()));  // tiny to 100
  // either side of every reduction boundary (y = (j + 1/2) ln2) and of k ln2
  for (int j = 0; j < 1100; ++j) {
    const double b = -(j + 0.5) * 0.6931471805599453, c = -j * 0.6931471805599453;
    for (int d = -40; d <= 40; ++d) {
      check(b + d * 1e-15 * (1.0 + j));
      check(c + d * 1e-15 * (1.0 + j));
    }
  }
  double ey, em;
  vrc::expd::exp_expm1(0.0, &ey, &em);
  const bool exact0 = ey == 1.0 && em == 0.0;
  vrc::expd::exp_expm1(-1e-300, &ey, &em);
  const bool tiny = ey == 1.0 && em == -1e-300;
  printf("checked %ld: worst exp %.3f ulp at y=%.17g, worst expm1 %.3f ulp at y=%.17g; "
         "below-range failures %ld; exact at 0: %d; tiny: %d\n",
         n_checked, worst_ey, at_ey, worst_em, at_em, n_bad_range, exact0, tiny);
  return (worst_ey <= 2.0 && worst_em <= 2.0 && n_bad_range == 0 && exact0 && tiny) ? 0 : 1;
}
