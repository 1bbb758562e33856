// Host-side check of the float-float helpers of the mixed path (compiled as host code):
// ff_to_double_rn, the integer conversion of a float-float pair to FP64, must give the bits of
// the FP64 addition hi + lo (round to nearest, ties to even) for every normalized pair, and
// ff_from_double / ff_add must be error-free where the transformations they use are.
// Prints the number of pairs checked and of mismatches; exits non-zero on a mismatch.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "fmg_ff.cuh"

using fmg::ff;

static ff two_sum_pair(float a, float b) {
  const float s = a + b, bb = s - a;
  return ff{s, (a - (s - bb)) + (b - bb)};
}

int main(int argc, char** argv) {
  const long long rounds = argc > 1 ? atoll(argv[1]) : 1000000;
  std::mt19937_64 rng(20161117);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::uniform_int_distribution<int> E(-60, 60), Gap(0, 80), Bit(0, 1);
  long long n = 0, bad = 0;
  auto check = [&](ff x) {
    const double want = (double)x.hi + (double)x.lo, got = fmg::ff_to_double_rn(x);
    uint64_t a, b;
    memcpy(&a, &want, 8);
    memcpy(&b, &got, 8);
    ++n;
    if (a != b && !(std::isnan(want) && std::isnan(got))) {
      if (bad < 5) printf("mismatch: hi=%a lo=%a add=%a int=%a\n", x.hi, x.lo, want, got);
      ++bad;
    }
  };
  for (long long i = 0; i < rounds; ++i) {
    // a double split into a pair (the path's conversion from FP64)
    const double x = std::ldexp(U(rng), E(rng));
    const ff f = fmg::ff_from_double(x);
    check(f);
    if ((double)f.hi + (double)f.lo != x && std::fabs(x) > 1e-30) {
      // a double with more than 48 significant bits is rounded by the split: it must be within
      // 2^-48 relative
      if (std::fabs(((double)f.hi + (double)f.lo - x) / x) > std::ldexp(1.0, -47)) ++bad;
    }
    // error-free sums of two floats over a range of exponent gaps: exact pairs, ties, cancellation
    check(two_sum_pair((float)std::ldexp(U(rng), E(rng)), (float)std::ldexp(U(rng), E(rng) - Gap(rng))));
    // hi a power of two with lo of either sign (the borrow case)
    const int k = E(rng);
    check(two_sum_pair(std::ldexp(1.0f, k) * (Bit(rng) ? 1.f : -1.f), std::ldexp(1.0f, k - 24 - Gap(rng) / 8) * (float)U(rng)));
    // hi with an all-ones significand and lo = +-ulp(hi)/2 (the round-half and carry cases)
    check(two_sum_pair(std::nextafter(std::ldexp(1.0f, k + 1), 0.f), std::ldexp(1.0f, k - 24) * (Bit(rng) ? 1.f : -1.f)));
  }
  const float sp[] = {0.f, -0.f, 1e-40f, -1e-40f, INFINITY, -INFINITY, NAN, 1.f, -1.f, 3.4e38f, 1.2e-38f};
  for (float a : sp)
    for (float b : sp) {
      check(two_sum_pair(a, b * 1e-10f));
      check(ff{a, 0.f});
    }
  printf("%lld %lld\n", n, bad);
  return bad != 0;
}
