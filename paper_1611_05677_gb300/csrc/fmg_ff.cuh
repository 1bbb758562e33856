// Float-float ("double-single") arithmetic for the mixed-precision path.
//
// A value is an unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about 48
// significant bits.  The operations are built from the error-free transformations of
// Dekker (1971) and Knuth (TAOCP vol. 2, 4.2.2): TwoSum gives s + e = a + b exactly with
// s = fl(a + b); with a fused multiply-add, TwoProduct gives p + e = a * b exactly with
// p = fl(a * b).  On this GPU an FP32 operation issues 64 times as fast as an FP64 one, so a
// dozen FP32 operations per float-float step still cost a fraction of one FP64 operation.
// The path's FP64 quantities that feed sums over many nodes (residuals, moment sums) keep
// ~1e-14 relative accuracy this way, far below the discretization error that bounds the
// mixed path.
#pragma once

#include <cuda_runtime.h>

#include <cstring>

#include "fmg_internal.cuh"

namespace fmg {

struct ff {
  float hi, lo;
};

// s + e = a + b exactly (s = fl(a + b)).
__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// s + e = a + b exactly when |a| >= |b| or a = 0.
__host__ __device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

// p + e = a * b exactly (p = fl(a * b)), with one fused multiply-add.
__host__ __device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

__host__ __device__ __forceinline__ ff ff_make(float hi, float lo) {
  ff r;
  quick_two_sum(hi, lo, r.hi, r.lo);
  return r;
}

// x + y, accurate also under cancellation (both parts through TwoSum).
__host__ __device__ __forceinline__ ff ff_add(ff x, ff y) {
  float s, e, t, f;
  two_sum(x.hi, y.hi, s, e);
  two_sum(x.lo, y.lo, t, f);
  e += t;
  quick_two_sum(s, e, s, e);
  e += f;
  ff r;
  quick_two_sum(s, e, r.hi, r.lo);
  return r;
}

// x + y for accumulating sums: the lo parts are added without their own TwoSum, so the error
// is bounded relative to |x| + |y| (as for an FP64 add) rather than to |x + y|.
__host__ __device__ __forceinline__ ff ff_add_fast(ff x, ff y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  e += x.lo + y.lo;
  ff r;
  quick_two_sum(s, e, r.hi, r.lo);
  return r;
}

__host__ __device__ __forceinline__ ff ff_neg(ff x) { return ff{-x.hi, -x.lo}; }
__host__ __device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

// x + b for an FP32 b.
__host__ __device__ __forceinline__ ff ff_add_f(ff x, float b) {
  float s, e;
  two_sum(x.hi, b, s, e);
  e += x.lo;
  ff r;
  quick_two_sum(s, e, r.hi, r.lo);
  return r;
}

// x * y (the lo * lo term, below the format's precision, is dropped).
__host__ __device__ __forceinline__ ff ff_mul(ff x, ff y) {
  float p, e;
  two_prod(x.hi, y.hi, p, e);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  ff r;
  quick_two_sum(p, e, r.hi, r.lo);
  return r;
}

// x * b for an FP32 b.
__host__ __device__ __forceinline__ ff ff_mul_f(ff x, float b) {
  float p, e;
  two_prod(x.hi, b, p, e);
  e = fmaf(x.lo, b, e);
  ff r;
  quick_two_sum(p, e, r.hi, r.lo);
  return r;
}

// Conversions.  From FP64: hi = fl32(x), lo = fl32(x - hi) (x - hi is exact in FP64).
__host__ __device__ __forceinline__ ff ff_from_double(double x) {
  ff r;
  r.hi = (float)x;
  r.lo = (float)(x - (double)r.hi);
  return r;
}
__host__ __device__ __forceinline__ double ff_to_double(ff x) { return (double)x.hi + (double)x.lo; }

__host__ __device__ __forceinline__ unsigned ff_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ double ff_double_from_bits(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
#endif
}

// hi + lo rounded to the nearest double (ties to even), the value ff_to_double gives, formed
// with integer operations only: this GPU issues FP64 instructions (conversions included) at
// 1/64 of the FP32 rate, and a pass that writes an FP64 result per node is otherwise bound by
// them.  From the IEEE-754 binary32/binary64 formats: for a pair with hi normal, lo normal or
// zero and |lo| <= ulp(hi)/2, the significands are aligned on a 64-bit integer (hi's leading
// bit at bit 62), added or subtracted with a sticky bit for the bits of lo shifted out,
// normalized by at most one place and rounded at bit 10.  Zero, subnormal, infinite and NaN
// parts take the FP64 add.
__host__ __device__ __forceinline__ double ff_to_double_rn(ff x) {
  const unsigned bh = ff_bits(x.hi), bl = ff_bits(x.lo);
  const int eh = (int)((bh >> 23) & 0xffu), el = (int)((bl >> 23) & 0xffu);
  const unsigned long long sign = (unsigned long long)(bh >> 31) << 63;
  const int d = eh - el;
  const bool lo_zero = (bl & 0x7fffffffu) == 0u;
  if (eh == 0 || eh == 255 || (!lo_zero && (el == 0 || d < 24))) return ff_to_double(x);
  const unsigned long long H = (unsigned long long)((bh & 0x7fffffu) | 0x800000u);
  if (lo_zero) return ff_double_from_bits(sign | ((unsigned long long)(eh + 896) << 52) | ((H & 0x7fffffull) << 29));
  const unsigned long long Lm = (unsigned long long)((bl & 0x7fffffu) | 0x800000u);
  // lo on hi's grid: hi = H 2^(eh-150) = (H << 39) 2^(eh-189); lo = Lm 2^(el-150) = (Lm << (39-d)) 2^(eh-189)
  unsigned long long L;
  bool sticky = false;
  if (d <= 39) {
    L = Lm << (39 - d);
  } else if (d < 64) {
    L = Lm >> (d - 39);
    sticky = (Lm & ((1ull << (d - 39)) - 1ull)) != 0ull;
  } else {
    L = 0ull;
    sticky = true;
  }
  unsigned long long R = H << 39;
  int e = eh + 896;                                 // double exponent field of 2^(eh-127)
  if (((bh ^ bl) >> 31) == 0u) {
    R += L;                                         // true value: R + (a fraction if sticky)
  } else {
    R -= L;
    if (sticky) R -= 1ull;                          // true value: R + a fraction in (0, 1)
  }
  if (R >> 63) {                                    // carried past bit 62
    sticky = sticky || (R & 1ull);
    R >>= 1;
    ++e;
  } else if (!(R >> 62)) {                          // borrowed below bit 62 (at most one place)
    R <<= 1;
    --e;
  }
  unsigned long long m = R >> 10;                   // 53 significant bits
  const bool round = (R >> 9) & 1ull;
  sticky = sticky || (R & 0x1ffull) != 0ull;
  if (round && (sticky || (m & 1ull))) {
    ++m;
    if (m >> 53) {
      m >>= 1;
      ++e;
    }
  }
  return ff_double_from_bits(sign | ((unsigned long long)e << 52) | (m & 0xfffffffffffffull));
}

// The exact FP64 value of an FP32 number, built from its bits for normal numbers and zeros
// (sign; exponent rebiased from 127 to 1023, i.e. + 896; significand moved up by 29 places), so
// that no FP64 conversion instruction is issued; subnormal, infinite and NaN inputs take the
// conversion.
__host__ __device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned b = ff_bits(f);
  const unsigned e = (b >> 23) & 0xffu;
  if ((b & 0x7fffffffu) == 0u) return ff_double_from_bits((unsigned long long)(b >> 31) << 63);
  if (e == 0u || e == 255u) return (double)f;
  const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  const unsigned lo = b << 29;
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  return ff_double_from_bits(((unsigned long long)hi << 32) | lo);
#endif
}

// hi + lo rounded to the nearest double: the two exact conversions above and one FP64 add, the
// value ff_to_double gives with one FP64 instruction per pair instead of three.
__host__ __device__ __forceinline__ double ff_to_double_fast(ff x) {
  return f32_to_f64_bits(x.hi) + f32_to_f64_bits(x.lo);
}

// A float-float value stored in an 8-byte slot (the layout of the double arrays it replaces).
__device__ __forceinline__ ff ff_load(const double* p) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  return ff{v.x, v.y};
}
__device__ __forceinline__ void ff_store(double* p, ff x) { *reinterpret_cast<float2*>(p) = make_float2(x.hi, x.lo); }

// sum_k (u_k - u_c) over the 2d axis neighbours of a node with value uc, from the neighbour
// values um[ax] (at -1 along axis ax) and up[ax] (at +1): the hi differences and their sum
// through TwoSum (exact), the lo parts and the rounding terms added after.
template <int D>
__host__ __device__ __forceinline__ ff neighbour_sum_ff_v(ff uc, const ff* um, const ff* up) {
  float s = 0.f, lo = 0.f;
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int ax = 0; ax < D; ++ax) {
    float dm, em, dp, ep, t, et;
    two_sum(um[ax].hi, -uc.hi, dm, em);
    two_sum(up[ax].hi, -uc.hi, dp, ep);
    two_sum(dm, dp, t, et);
    float s2, e2;
    two_sum(s, t, s2, e2);
    s = s2;
    lo += ((em + ep) + (et + e2)) + ((um[ax].lo - uc.lo) + (up[ax].lo - uc.lo));
  }
  ff r;
  two_sum(s, lo, r.hi, r.lo);
  return r;
}

// The variable-coefficient form (VarCoef, A(x) != I): sum_e w_e (u_e - u_c) over the 2d axis
// edges, nb[] in the order x-, x+, y-, y+ (, z-, z+); the differences are formed exactly (TwoSum
// on the leading parts), weighted by the float-float edge sums of the coefficient table and
// summed in float-float, and the total is scaled by the weights' common factor (1/2 in 2D,
// 1/6 in 3D).
template <int D>
__device__ __forceinline__ ff weighted_neighbour_sum_ff(ff uc, const ff* nb, const VarCoef& vc, int ls, int i, int j,
                                                        int l) {
  ff W[2 * D];
  edge_weights<D, ff>(
      vc.nc, ls, i, j, l,
      [&](int k) {
        const float2 v = *reinterpret_cast<const float2*>(vc.aff + k);
        return ff{v.x, v.y};
      },
      [](ff a, ff b) { return ff_add(a, b); }, [](ff x) { return x; }, W);
  ff S{0.f, 0.f};
#pragma unroll
  for (int e = 0; e < 2 * D; ++e) {
    float dh, de;
    two_sum(nb[e].hi, -uc.hi, dh, de);
    ff d;
    quick_two_sum(dh, de + (nb[e].lo - uc.lo), d.hi, d.lo);
    S = ff_add(S, ff_mul(d, W[e]));
  }
  if (D == 2) return ff{0.5f * S.hi, 0.5f * S.lo};
  return ff_mul(S, ff{0x1.555556p-3f, -0x1.555556p-28f});   // x 1/6
}

// The same at node c of a nodal array (axis strides 1, np, pl).
template <int D>
__device__ __forceinline__ ff neighbour_sum_ff(const double* __restrict__ u, long long c, long long np, long long pl) {
  const long long o[3] = {1, np, pl};
  ff um[D], up[D];
#pragma unroll
  for (int ax = 0; ax < D; ++ax) {
    um[ax] = ff_load(u + c - o[ax]);
    up[ax] = ff_load(u + c + o[ax]);
  }
  return neighbour_sum_ff_v<D>(ff_load(u + c), um, up);
}

// 2^k x for an integer k with |k| <= 126 (exact unless the parts underflow).
__host__ __device__ __forceinline__ ff ff_ldexp(ff x, int k) {
  const float sc = ldexpf(1.0f, k);
  return ff{x.hi * sc, x.lo * sc};
}

// exp(x) - 1 in float-float, from the exponential's own properties: x = k ln2 + r with k the
// nearest integer to x / ln2 (|r| <= ln2 / 2, r formed in float-float with ln2 split into two
// FP32 parts), then r = 2^5 s with |s| <= 0.011, expm1(s) by its Taylor series through s^6 (the
// next term is below 4e-18), five squarings in the form q <- q (2 + q) (that is (1+q)^2 - 1,
// which keeps the relative accuracy of a small q), and expm1(x) = 2^k q + (2^k - 1).  Relative
// error about 1e-13 over the range the nonlinearities meet; |x| beyond 80 returns the FP32
// limit (exp overflows there in FP32 anyway).
__host__ __device__ __forceinline__ ff ff_expm1(ff x) {
  // the float-float split hi = fl32(c), lo = fl32(c - hi) of the constants, as exact hex literals
  const float kLn2Hi = 0x1.62e430p-1f, kLn2Lo = -0x1.05c610p-29f;   // ln 2
  const float kInvLn2 = 0x1.715476p+0f;                                // fl32(1 / ln 2)
  if (!(x.hi > -80.f && x.hi < 80.f)) {
    const float e = expm1f(x.hi);
    return ff{e, 0.f};
  }
  const float kf = rintf(x.hi * kInvLn2);
  const int k = (int)kf;
  // r = x - k ln2: both products exact (TwoProduct), then float-float sums
  float p1, e1, p2, e2;
  two_prod(kf, kLn2Hi, p1, e1);
  two_prod(kf, kLn2Lo, p2, e2);
  ff r = ff_add(x, ff{-p1, -e1});
  r = ff_add(r, ff{-p2, -e2});
  const ff sx = ff_ldexp(r, -5);
  // Taylor series of expm1 at s: s (1 + s (1/2 + s (1/6 + s (1/24 + s (1/120 + s / 720)))))
  const ff c720 = ff{0x1.6c16c2p-10f, -0x1.27d27ep-35f};   // 1/720
  const ff c120 = ff{0x1.111112p-7f, -0x1.dddddep-32f};   // 1/120
  const ff c24 = ff{0x1.555556p-5f, -0x1.555556p-30f};     // 1/24
  const ff c6 = ff{0x1.555556p-3f, -0x1.555556p-28f};      // 1/6
  ff q = ff_add(ff_mul(c720, sx), c120);
  q = ff_add(ff_mul(q, sx), c24);
  q = ff_add(ff_mul(q, sx), c6);
  q = ff_add(ff_mul(q, sx), ff{0.5f, 0.f});
  q = ff_add(ff_mul(q, sx), ff{1.f, 0.f});
  q = ff_mul(q, sx);
#pragma unroll
  for (int i = 0; i < 5; ++i) q = ff_mul(q, ff_add_f(q, 2.0f));
  if (k == 0) return q;
  // 2^k (1 + q) - 1 = 2^k q + (2^k - 1); 2^k - 1 is exact in FP32 for |k| <= 24
  const float pk = ldexpf(1.0f, k) - 1.0f;
  if (k >= -24 && k <= 24) return ff_add(ff_ldexp(q, k), ff{pk, 0.f});
  return ff_add_f(ff_ldexp(q, k), pk);
}

// sqrt(x) for x >= 0 in float-float: the FP32 root s, then one Newton step
// s + (x - s^2) / (2 s) with the residual x - s^2 formed exactly (TwoProduct).
__host__ __device__ __forceinline__ ff ff_sqrt(ff x) {
  if (!(x.hi > 0.f)) return ff{0.f, 0.f};
  const float s = sqrtf(x.hi);
  float p, e;
  two_prod(s, s, p, e);
  const ff res = ff_add(x, ff{-p, -e});
  const float corr = (res.hi + res.lo) / (2.0f * s);
  ff r;
  quick_two_sum(s, corr, r.hi, r.lo);
  return r;
}

__host__ __device__ __forceinline__ ff ff_abs(ff x) { return x.hi < 0.f ? ff_neg(x) : x; }

// a f(u) in float-float for the nonlinearities of Sec. 4 (the mixed path's per-node f, which
// enters the residual sums): polynomial ones directly, the exponential ones through ff_expm1,
// sign(u)|u|^{3/2} through ff_sqrt.
__device__ __forceinline__ ff f_ff(int kind, ff a, double a64, ff u) {
  (void)a64;
  switch (kind) {
    case FMG_F_CUBIC: return ff_mul(ff_mul(ff_mul(u, u), u), a);
    case FMG_F_LINEAR: return ff_mul(u, a);
    case FMG_F_EXPM1: return ff_mul(ff_expm1(u), a);
    case FMG_F_NEG_EXP_NEG: return ff_neg(ff_mul(ff_add_f(ff_expm1(ff_neg(u)), 1.0f), a));   // -a (expm1(-u) + 1)
    default: return ff_mul(ff_mul(u, ff_sqrt(ff_abs(u))), a);                                   // a u |u|^{1/2}
  }
}

}  // namespace fmg
