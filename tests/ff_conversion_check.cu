// Host-side check of the float-float helpers of the mixed path (compiled as host code).
// ff_to_double_rn, the integer conversion of a float-float pair to FP64, and ff_to_double_fast,
// the conversion through FP64 values built from the FP32 bits, must give the bits of the FP64
// addition hi + lo (round to nearest, ties to even) for every normalized pair.  The
// error-free transformations must be exact: two_sum gives s + e = a + b and two_prod gives
// p + e = a b, checked in FP64 where these sums are exact.  The float-float operations must stay
// within their error bounds, checked against quad-precision sums of the float parts (113 bits hold every sum here exactly): ff_add
// within 2^-44 |x + y| (also under cancellation), ff_add_fast within 2^-44 (|x| + |y|), ff_mul
// within 2^-44 |x y|, and the stencil neighbour sum within 2^-42 of its largest input.  The
// float-float expm1 and sqrt of the nonlinearities are checked against the host's FP64 functions.
// Prints the number of conversion pairs checked and the number of failed checks; exits
// non-zero on a failure.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "fmg_ff.cuh"

using fmg::ff;
// quad precision, the exact reference of the float-float bounds: IEEE binary128 is long double
// on AArch64 and GCC's __float128 on x86-64
#if defined(__aarch64__)
typedef long double Q;
#else
typedef __float128 Q;
#endif
static Q qabs(Q x) { return x < 0 ? -x : x; }

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
    const double got2 = fmg::ff_to_double_fast(x);
    uint64_t a, b, c;
    memcpy(&a, &want, 8);
    memcpy(&b, &got, 8);
    memcpy(&c, &got2, 8);
    ++n;
    if (a != b && !(std::isnan(want) && std::isnan(got))) {
      if (bad < 5) printf("mismatch: hi=%a lo=%a add=%a int=%a\n", x.hi, x.lo, want, got);
      ++bad;
    }
    if (a != c && !(std::isnan(want) && std::isnan(got2))) {
      if (bad < 5) printf("mismatch: hi=%a lo=%a add=%a bits+add=%a\n", x.hi, x.lo, want, got2);
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
  // error-free transformations and float-float error bounds (moderate exponents: no underflow)
  std::uniform_int_distribution<int> Em(-20, 20), Small(0, 28);
  auto rf = [&](int e) { return (float)std::ldexp(U(rng), e); };
  auto rff = [&](int e) { return fmg::ff_from_double(std::ldexp(U(rng), e)); };
  auto ld = [](ff x) { return (Q)x.hi + (Q)x.lo; };
  auto fail = [&](const char* what, double err, double bound) {
    if (bad < 5) printf("%s: error %g above %g\n", what, err, bound);
    ++bad;
  };
  const double u44 = std::ldexp(1.0, -44), u42 = std::ldexp(1.0, -42);
  for (long long i = 0; i < rounds; ++i) {
    const int e = Em(rng);
    const float a = rf(e), b = rf(e - Small(rng));
    float s, t;
    fmg::two_sum(a, b, s, t);
    if (s != a + b || (double)s + (double)t != (double)a + (double)b) fail("two_sum", std::fabs((double)s + t - ((double)a + b)), 0);
    fmg::two_prod(a, b, s, t);
    if (s != a * b || (double)s + (double)t != (double)a * (double)b) fail("two_prod", std::fabs((double)s + t - (double)a * b), 0);
    const ff x = rff(e), y = Bit(rng) ? rff(e - Small(rng)) : ff{-x.hi, -x.lo * (float)U(rng)};   // cancellation too
    const Q xs = ld(x), ys = ld(y);
    const Q sum = xs + ys;
    const double e_add = (double)qabs(ld(fmg::ff_add(x, y)) - sum);
    if (e_add > u44 * (double)qabs(sum) && e_add > 0) fail("ff_add", e_add, u44 * (double)qabs(sum));
    const double e_fast = (double)qabs(ld(fmg::ff_add_fast(x, y)) - sum);
    if (e_fast > u44 * (double)(qabs(xs) + qabs(ys))) fail("ff_add_fast", e_fast, u44 * (double)(qabs(xs) + qabs(ys)));
    const double e_mul = (double)qabs(ld(fmg::ff_mul(x, y)) - xs * ys);
    if (e_mul > u44 * (double)qabs(xs * ys)) fail("ff_mul", e_mul, u44 * (double)qabs(xs * ys));
    // sum over the 2d axis neighbours of (u_k - u_c), values of one magnitude as on a smooth grid
    ff uc = rff(0), um[3], up[3];
    Q exact = 0, big = qabs(ld(uc));
    for (int ax = 0; ax < 3; ++ax) {
      um[ax] = fmg::ff_from_double((double)ld(uc) + std::ldexp(U(rng), -Small(rng)));
      up[ax] = fmg::ff_from_double((double)ld(uc) + std::ldexp(U(rng), -Small(rng)));
      exact += (ld(um[ax]) - ld(uc)) + (ld(up[ax]) - ld(uc));
      big = std::max(big, std::max(qabs(ld(um[ax])), qabs(ld(up[ax]))));
    }
    const double e_nb = (double)qabs(ld(fmg::neighbour_sum_ff_v<3>(uc, um, up)) - exact);
    if (e_nb > u42 * (double)big) fail("neighbour_sum_ff_v", e_nb, u42 * (double)big);
  }
  // the float-float exponential and root of the mixed path's nonlinearities, against the host's
  // long-double expm1 and FP64 sqrt (errors far below the bounds checked): expm1 within 2^-45
  // relative over [-12, 12] (small arguments included, where expm1 keeps its relative accuracy,
  // and arguments next to the multiples of ln2/64 where its table index changes), sqrt within
  // 2^-44 relative; and the tables 2^(j/64), 2^(j/64) - 1 within 2^-48 of long-double exp2
  for (int j = -32; j < 32; ++j) {
    const ff t = fmg::exp2_64(j + 32), m = fmg::exp2m1_64(j + 32);
    const long double v = exp2l((long double)j / 64);
    const long double et = fabsl((long double)t.hi + (long double)t.lo - v);
    if (et > std::ldexp(1.0L, -48) * v) fail("exp2_64 table", (double)et, std::ldexp(1.0, -48));
    const long double em = fabsl((long double)m.hi + (long double)m.lo - (v - 1));
    if (em > std::ldexp(1.0L, -48) * fabsl(v - 1)) fail("exp2m1_64 table", (double)em, std::ldexp(1.0, -48));
  }
  std::uniform_real_distribution<double> X(-12.0, 12.0);
  const double u45r = std::ldexp(1.0, -45);
  for (long long i = 0; i < rounds / 4; ++i) {
    double x = X(rng);
    if (i % 3 == 1) x = std::ldexp(U(rng), -Small(rng)) * ((i & 4) ? -1.0 : 1.0);   // small arguments
    if (i % 5 == 2) x = (double)(i % 2001 - 1000) * 0.010830424696249145 + std::ldexp(U(rng) - 0.5, -14);
    const ff fx = fmg::ff_from_double(x);
    const long double xe = (long double)fx.hi + (long double)fx.lo;    // the argument as represented
    const long double want = expm1l(xe);
    const ff ge = fmg::ff_expm1(fx);
    const long double got = (long double)ge.hi + (long double)ge.lo;
    if (fabsl(got - want) > u45r * fabsl(want))
      fail("ff_expm1", (double)fabsl(got - want), u45r * (double)fabsl(want));
    const double ax = std::fabs((double)xe) * 7.0;
    const ff fa = fmg::ff_from_double(ax);
    const double wr = std::sqrt((double)fa.hi + (double)fa.lo);
    const ff r = fmg::ff_sqrt(fa);
    const double gr = (double)r.hi + (double)r.lo;
    if (std::fabs(gr - wr) > u44 * wr) fail("ff_sqrt", std::fabs(gr - wr), u44 * wr);
  }
  if (fmg::ff_expm1(ff{0.f, 0.f}).hi != 0.f) fail("ff_expm1(0)", 1.0, 0.0);
  const float sp[] = {0.f, -0.f, 1e-40f, -1e-40f, INFINITY, -INFINITY, NAN, 1.f, -1.f, 3.4e38f, 1.2e-38f};
  for (float a : sp)
    for (float b : sp) {
      check(two_sum_pair(a, b * 1e-10f));
      check(ff{a, 0.f});
    }
  printf("%lld %lld\n", n, bad);
  return bad != 0;
}
