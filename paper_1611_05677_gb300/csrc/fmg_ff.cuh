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

// 2^(j/64) for j = -32 .. 31 (row j + 32) and 2^(j/64) - 1, as float-float pairs (hi = fl32(v),
// lo = fl32(v - hi)), evaluated in 60-digit decimal arithmetic; the host check compares them with
// the host's long-double exp2.
#define FMG_EXP2_64 \
  { \
      {0x1.6a09e6p-1f, 0x1.9fcef4p-27f}, {0x1.6dfb24p-1f, -0x1.cd72e8p-28f}, {0x1.71f75ep-1f, 0x1.1d8beep-26f}, \
      {0x1.75feb6p-1f, -0x1.37b306p-26f}, {0x1.7a1148p-1f, -0x1.829fdp-26f}, {0x1.7e2f34p-1f, -0x1.261634p-26f}, \
      {0x1.82589ap-1f, -0x1.accc7cp-27f}, {0x1.868d9ap-1f, -0x1.2edb44p-27f}, {0x1.8ace54p-1f, 0x1.15506ep-28f}, \
      {0x1.8f1aeap-1f, -0x1.baa232p-27f}, {0x1.93737cp-1f, -0x1.e64744p-26f}, {0x1.97d82ap-1f, -0x1.0d8d84p-32f}, \
      {0x1.9c4918p-1f, 0x1.51f848p-28f}, {0x1.a0c668p-1f, -0x1.2886a6p-27f}, {0x1.a5503cp-1f, -0x1.b83b54p-26f}, \
      {0x1.a9e6b6p-1f, -0x1.50c048p-26f}, {0x1.ae89fap-1f, -0x1.a94b14p-27f}, {0x1.b33a2cp-1f, -0x1.ec3a82p-27f}, \
      {0x1.b7f77p-1f, -0x1.a09438p-26f}, {0x1.bcc1eap-1f, -0x1.f687c6p-26f}, {0x1.c199bep-1f, -0x1.3d56b2p-28f}, \
      {0x1.c67f12p-1f, 0x1.cafa2ap-26f}, {0x1.cb720ep-1f, -0x1.8837ccp-28f}, {0x1.d072d4p-1f, 0x1.40f13p-26f}, \
      {0x1.d5818ep-1f, -0x1.822dbcp-28f}, {0x1.da9e6p-1f, 0x1.ed9942p-28f}, {0x1.dfc974p-1f, -0x1.908c94p-26f}, \
      {0x1.e502eep-1f, 0x1.e2cffep-27f}, {0x1.ea4afap-1f, 0x1.52486cp-28f}, {0x1.efa1bep-1f, 0x1.cc2b44p-26f}, \
      {0x1.f50766p-1f, -0x1.246ebp-27f}, {0x1.fa7c18p-1f, 0x1.9e90d8p-29f}, {0x1p+0f, 0.0f}, \
      {0x1.02c9a4p+0f, -0x1.887fap-28f}, {0x1.059b0ep+0f, -0x1.9d4f52p-25f}, {0x1.087452p+0f, -0x1.e2990ep-26f}, \
      {0x1.0b5586p+0f, 0x1.9f3122p-25f}, {0x1.0e3ec4p+0f, -0x1.a585ccp-25f}, {0x1.11301ep+0f, -0x1.fdb496p-25f}, \
      {0x1.1429aap+0f, 0x1.d525bcp-25f}, {0x1.172b84p+0f, -0x1.c15742p-27f}, {0x1.1a35bep+0f, 0x1.6df96ep-25f}, \
      {0x1.1d4874p+0f, -0x1.d2e8cap-25f}, {0x1.2063b8p+0f, 0x1.0c519ap-25f}, {0x1.2387a6p+0f, 0x1.ceac48p-25f}, \
      {0x1.26b456p+0f, 0x1.789f38p-26f}, {0x1.29e9ep+0f, -0x1.5c0424p-25f}, {0x1.2d285ap+0f, 0x1.b900c2p-26f}, \
      {0x1.306fep+0f, 0x1.4636e2p-25f}, {0x1.33c08cp+0f, -0x1.b37d2p-25f}, {0x1.371a74p+0f, -0x1.18aac6p-25f}, \
      {0x1.3a7db4p+0f, -0x1.634c02p-25f}, {0x1.3dea64p+0f, 0x1.824684p-25f}, {0x1.4160a2p+0f, 0x1.f72e2ap-28f}, \
      {0x1.44e086p+0f, 0x1.8624b4p-30f}, {0x1.486a2cp+0f, -0x1.47d866p-25f}, {0x1.4bfdaep+0f, -0x1.593abcp-25f}, \
      {0x1.4f9b28p+0f, -0x1.2c5a6cp-25f}, {0x1.5342b6p+0f, -0x1.2c561p-25f}, {0x1.56f474p+0f, -0x1.295b04p-25f}, \
      {0x1.5ab07ep+0f, -0x1.5bd5ecp-27f}, {0x1.5e76f2p+0f, -0x1.4a5bd6p-25f}, {0x1.6247ecp+0f, -0x1.f8b55p-25f}, \
      {0x1.662388p+0f, 0x1.2a9112p-27f} \
  }
#define FMG_EXP2M1_64 \
  { \
      {-0x1.2bec34p-2f, 0x1.9fcef4p-27f}, {-0x1.2409b8p-2f, -0x1.cd72e8p-28f}, {-0x1.1c1142p-2f, -0x1.c4e824p-27f}, \
      {-0x1.140296p-2f, 0x1.9099f2p-27f}, {-0x1.0bdd72p-2f, 0x1.f580c4p-28f}, {-0x1.03a19ap-2f, 0x1.b3d398p-27f}, \
      {-0x1.f69d9ap-3f, 0x1.4cce12p-29f}, {-0x1.e5c99ap-3f, 0x1.a24976p-28f}, {-0x1.d4c6bp-3f, 0x1.15506ep-28f}, \
      {-0x1.c3945ap-3f, 0x1.157736p-29f}, {-0x1.b23214p-3f, 0x1.9b8bcap-30f}, {-0x1.a09f58p-3f, -0x1.0d8d84p-32f}, \
      {-0x1.8edbap-3f, 0x1.51f848p-28f}, {-0x1.7ce662p-3f, 0x1.aef2b2p-28f}, {-0x1.6abf14p-3f, 0x1.1f12aep-28f}, \
      {-0x1.58652ap-3f, -0x1.43012p-28f}, {-0x1.45d81ap-3f, 0x1.5ad3aep-29f}, {-0x1.331752p-3f, 0x1.3c57ecp-31f}, \
      {-0x1.202244p-3f, 0x1.7daf24p-28f}, {-0x1.0cf85cp-3f, 0x1.2f0748p-31f}, {-0x1.f33212p-4f, 0x1.85529cp-29f}, \
      {-0x1.cc0768p-4f, -0x1.a82eb4p-29f}, {-0x1.a46f92p-4f, 0x1.df20d2p-30f}, {-0x1.7c695ap-4f, -0x1.f87684p-29f}, \
      {-0x1.53f392p-4f, 0x1.f7490ep-30f}, {-0x1.2b0cfep-4f, -0x1.266bd4p-32f}, {-0x1.01b466p-4f, -0x1.08c942p-30f}, \
      {-0x1.afd118p-5f, -0x1.d30028p-31f}, {-0x1.5b505ep-5f, 0x1.4921b4p-30f}, {-0x1.05e412p-5f, 0x1.85689ep-31f}, \
      {-0x1.5f134ap-6f, 0x1.b91502p-31f}, {-0x1.60f9fap-7f, 0x1.e90d82p-33f}, {0.0f, 0.0f}, \
      {0x1.64d1f4p-7f, -0x1.0ff3e2p-33f}, {0x1.66c34cp-6f, 0x1.585744p-32f}, {0x1.0e8a3p-5f, 0x1.d66f2p-30f}, \
      {0x1.6ab0dap-5f, -0x1.9dbc28p-34f}, {0x1.c7d866p-5f, -0x1.6172fp-31f}, {0x1.1301dp-4f, 0x1.25b50ap-32f}, \
      {0x1.429aaep-4f, 0x1.525bcp-29f}, {0x1.72b83cp-4f, 0x1.f545ecp-30f}, {0x1.a35becp-4f, -0x1.206916p-29f}, \
      {0x1.d48732p-4f, -0x1.2e8cacp-29f}, {0x1.031dc4p-3f, 0x1.8a3358p-30f}, {0x1.1c3d38p-3f, -0x1.8a9dc8p-28f}, \
      {0x1.35a2b2p-3f, 0x1.e27cdep-28f}, {0x1.4f4efap-3f, 0x1.1fdee2p-28f}, {0x1.6942d4p-3f, -0x1.1bfcf4p-28f}, \
      {0x1.837f06p-3f, -0x1.ce48eap-28f}, {0x1.9e045ap-3f, -0x1.9be9p-28f}, {0x1.b8d39cp-3f, -0x1.8aac6ap-29f}, \
      {0x1.d3ed9ap-3f, 0x1.cb3feep-29f}, {0x1.ef5326p-3f, 0x1.234224p-32f}, {0x1.058288p-2f, 0x1.f72e2ap-28f}, \
      {0x1.138218p-2f, 0x1.8624b4p-30f}, {0x1.21a8aep-2f, -0x1.1f6198p-27f}, {0x1.2ff6b6p-2f, -0x1.64eaecp-27f}, \
      {0x1.3e6c9ep-2f, -0x1.62d35ap-28f}, {0x1.4d0ad6p-2f, -0x1.62b07ep-28f}, {0x1.5bd1cep-2f, -0x1.4ad826p-28f}, \
      {0x1.6ac1f8p-2f, -0x1.5bd5ecp-27f}, {0x1.79dbc6p-2f, -0x1.296f5cp-27f}, {0x1.891facp-2f, 0x1.d2ac26p-31f}, \
      {0x1.988e2p-2f, 0x1.2a9112p-27f} \
  }
__device__ const float2 kExp2_64_d[64] = FMG_EXP2_64;
__device__ const float2 kExp2m1_64_d[64] = FMG_EXP2M1_64;
static const float2 kExp2_64_h[64] = FMG_EXP2_64;
static const float2 kExp2m1_64_h[64] = FMG_EXP2M1_64;

__host__ __device__ __forceinline__ ff exp2_64(int row) {
#ifdef __CUDA_ARCH__
  const float2 v = __ldg(&kExp2_64_d[row]);
#else
  const float2 v = kExp2_64_h[row];
#endif
  return ff{v.x, v.y};
}
__host__ __device__ __forceinline__ ff exp2m1_64(int row) {
#ifdef __CUDA_ARCH__
  const float2 v = __ldg(&kExp2m1_64_d[row]);
#else
  const float2 v = kExp2m1_64_h[row];
#endif
  return ff{v.x, v.y};
}

// exp(x) - 1 in float-float, from the exponential's own properties.  x = N ln2/64 + r with N
// the nearest integer to 64 x / ln2 (r formed in float-float from the two-part ln2/64 and exact
// products, |r| <= ln2/128) and N = 64 k + j, j in [-32, 31]; then
//   expm1(x) = 2^k ((2^(j/64) - 1) + 2^(j/64) expm1(r)) + (2^k - 1),
// with both 2^(j/64) and 2^(j/64) - 1 from the tables (so the bracket does not cancel: j
// centred on 0 keeps it within a factor 3 of 2^(j/64) (1 + expm1(r)) - 1), and expm1(r) =
// r + r^2 (1/2 + r/6 + r^2/24 + r^3/120) by its Taylor series (the next term is below 2^-47 |r|);
// only r, r^2 and r/6 need float-float, the rest of the bracket is FP32.  Relative error about
// 2^-46 over the range the nonlinearities meet; |x| beyond 80 returns the FP32 limit (exp
// overflows there in FP32 anyway).
__host__ __device__ __forceinline__ ff ff_expm1(ff x) {
  const float kInvL = 0x1.715476p+6f;                          // fl32(64 / ln 2)
  const float kLHi = 0x1.62e43p-7f, kLLo = -0x1.05c61p-35f;     // ln2 / 64 as float-float
  if (!(x.hi > -80.f && x.hi < 80.f)) {
    const float e = expm1f(x.hi);
    return ff{e, 0.f};
  }
  const float nf = rintf(x.hi * kInvL);
  const int N = (int)nf;
  const int k = (N + 32) >> 6;
  const int j = N - 64 * k;
  // r = x - N ln2/64: both products exact (TwoProduct), then float-float sums
  float p1, e1, p2, e2;
  two_prod(nf, kLHi, p1, e1);
  two_prod(nf, kLLo, p2, e2);
  ff r = ff_add(x, ff{-p1, -e1});
  r = ff_add(r, ff{-p2, -e2});
  const ff c6 = ff{0x1.555556p-3f, -0x1.555556p-28f};         // 1/6
  const float rh = r.hi;
  const float t = (rh * rh) * fmaf(rh, 0x1.111112p-7f, 0x1.555556p-5f);   // r^2 (1/24 + r/120)
  const ff B = ff_add_f(ff_add_f(ff_mul(r, c6), t), 0.5f);
  const ff q = ff_add_fast(r, ff_mul(ff_mul(r, r), B));          // expm1(r)
  const ff a = ff_add(exp2m1_64(j + 32), ff_mul(exp2_64(j + 32), q));
  if (k == 0) return a;
  // 2^k a + (2^k - 1); 2^k - 1 is exact in FP32 for |k| <= 24
  const float pk = ldexpf(1.0f, k) - 1.0f;
  if (k >= -24 && k <= 24) return ff_add(ff_ldexp(a, k), ff{pk, 0.f});
  return ff_add_f(ff_ldexp(a, k), pk);
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
