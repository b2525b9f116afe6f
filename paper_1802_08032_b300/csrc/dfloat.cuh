// Double-float ("df") arithmetic: a real number held as the unevaluated sum
// hi + lo of two floats, computed on the FP32 pipes.
//
// B300 runs FP32 about 58x faster than FP64 (65 vs 1.1 TFLOP/s measured),
// so complex128 tiles can be updated in df and converted to / from IEEE
// double only when a tile is loaded or stored.  Building blocks are the
// classic error-free transformations:
//   two_sum       (Knuth, TAOCP vol. 2):   s + e = a + b exactly
//   fast_two_sum  (Dekker 1971, |a|>=|b|): s + e = a + b exactly
//   two_prod      (FMA form):              p + e = a * b exactly
// Additions use the "sloppy" df sum (one two_sum on the high parts, low parts
// added in float, one renormalisation); its error is a few units of 2^-48 of
// the operands' magnitude, which bounds the absolute error of every update.
// Conversions: double -> df keeps the top 24 significand bits in hi and the
// next 29, rounded to 24, in lo (relative error <= 2^-47), computed with
// integer operations; df -> double converts hi and lo exactly and adds them
// with one FP64 addition.  Magnitudes below 2^-126 (hi) or 2^-74 (lo part)
// are flushed to zero: an absolute error below 1e-22 per amplitude.
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#include <cuda_runtime.h>
#endif

namespace qs {

struct df {
  float hi, lo;
};
struct dfc {
  df re, im;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// Sum of four df products a_k b_k, accumulated with exact high-part sums.
__device__ __forceinline__ df df_dot4(df a0, df b0, df a1, df b1, df a2, df b2, df a3, df b3) {
  const df A[4] = {a0, a1, a2, a3}, B[4] = {b0, b1, b2, b3};
  float s = 0.f, err = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float p = __fmul_rn(A[k].hi, B[k].hi);
    float e = __fmaf_rn(A[k].hi, B[k].hi, -p);
    e = __fmaf_rn(A[k].hi, B[k].lo, e);
    e = __fmaf_rn(A[k].lo, B[k].hi, e);
    if (k == 0) {
      s = p;
      err = e;
    } else {
      const df t = two_sum(s, p);
      s = t.hi;
      err = __fadd_rn(err, __fadd_rn(t.lo, e));
    }
  }
  return fast_two_sum(s, err);
}

__device__ __forceinline__ dfc dfc_add(dfc a, dfc b) { return dfc{df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ dfc dfc_sub(dfc a, dfc b) { return dfc{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }

// (c + i s) * v
__device__ __forceinline__ dfc dfc_mul(dfc v, df c, df s) {
  return dfc{df_sub(df_mul(c, v.re), df_mul(s, v.im)), df_add(df_mul(s, v.re), df_mul(c, v.im))};
}

// (ar + i ai) x + (br + i bi) y
__device__ __forceinline__ dfc dfc_mac2(df ar, df ai, dfc x, df br, df bi, dfc y) {
  return dfc{df_dot4(ar, x.re, df_neg(ai), x.im, br, y.re, df_neg(bi), y.im),
             df_dot4(ar, x.im, ai, x.re, br, y.im, bi, y.re)};
}

// IEEE double -> df (integer operations plus one int->float conversion).
__device__ __forceinline__ df df_from_double(double x) {
  const uint32_t hw = uint32_t(__double2hiint(x)), lw = uint32_t(__double2loint(x));
  const uint32_t sign = hw & 0x80000000u;
  const int e = int((hw >> 20) & 0x7FFu);  // biased exponent, 1023 = 2^0
  if (e < 897) return df{__uint_as_float(sign), __uint_as_float(sign)};  // |x| < 2^-126
  if (e > 1150) return df{float(x), 0.f};                                 // out of float range
  const uint32_t m23 = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  const float h = __uint_as_float(sign | (uint32_t(e - 896) << 23) | m23);
  float l = 0.f;
  if (e >= 949) {  // lo part = r 2^(e-1075) with r the 29 low significand bits
    const uint32_t r = lw & 0x1FFFFFFFu;
    l = __fmul_rn(__uint2float_rn(r), __uint_as_float(uint32_t(e - 948) << 23));
    l = __uint_as_float(__float_as_uint(l) | sign);
  }
  return df{h, l};
}

// Exact float -> double by bit manipulation (subnormal floats flush to 0).
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t sign = b & 0x80000000u, e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  if (e == 0) return __hiloint2double(int(sign), 0);
  if (e == 0xFF) return double(f);
  return __hiloint2double(int(sign | ((e + 896u) << 20) | (m >> 3)), int(m << 29));
}

__device__ __forceinline__ double df_to_double(df a) { return __dadd_rn(f2d_exact(a.hi), f2d_exact(a.lo)); }

}  // namespace qs

// ------------------------------------------------------------------------
// Packed complex double-float: hi = (re.hi, im.hi), lo = (re.lo, im.lo).
// The same error-free transformations, applied to the real and imaginary
// parts at once with the paired FP32 instructions of sm_100+ (one add /
// multiply / FMA on two floats per lane; each half rounds exactly as the
// scalar instruction would).
namespace qs {

struct dfc2 {
  float2 hi, lo;
};

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b with one rounding: (-1) * b is exact, the FMA rounds once.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ dfc2 two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  const float2 bb = sub2(s, a);
  return dfc2{s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}

__device__ __forceinline__ dfc2 two_diff2(float2 a, float2 b) {
  const float2 s = sub2(a, b);
  const float2 bb = sub2(s, a);
  return dfc2{s, sub2(sub2(a, sub2(s, bb)), add2(b, bb))};
}

__device__ __forceinline__ dfc2 fast_two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  return dfc2{s, sub2(b, sub2(s, a))};
}

__device__ __forceinline__ dfc2 dfc2_add(dfc2 a, dfc2 b) {
  const dfc2 s = two_sum2(a.hi, b.hi);
  return fast_two_sum2(s.hi, add2(s.lo, add2(a.lo, b.lo)));
}

__device__ __forceinline__ dfc2 dfc2_sub(dfc2 a, dfc2 b) {
  const dfc2 s = two_diff2(a.hi, b.hi);
  return fast_two_sum2(s.hi, add2(s.lo, sub2(a.lo, b.lo)));
}

// Element-wise product with a packed df factor c = (c0, c1) (each half its
// own df number): (a.re * c0, a.im * c1).
__device__ __forceinline__ dfc2 dfc2_mulv(dfc2 a, float2 chi, float2 clo) {
  const float2 p = mul2(a.hi, chi);
  const float2 np = mul2(a.hi, f2(-chi.x, -chi.y));  // -p exactly
  float2 e = fma2(a.hi, chi, np);
  e = fma2(a.hi, clo, e);
  e = fma2(a.lo, chi, e);
  return fast_two_sum2(p, e);
}

// Multiplication by i: (re, im) -> (-im, re), a swap and a sign.
__device__ __forceinline__ dfc2 dfc2_swap(dfc2 a) { return dfc2{f2(a.hi.y, a.hi.x), f2(a.lo.y, a.lo.x)}; }

// (cr + i ci) * v for a complex df factor: cr (re, im) + ci (-im, re).
__device__ __forceinline__ dfc2 dfc2_cmul(dfc2 v, df cr, df ci) {
  const dfc2 a = dfc2_mulv(v, f2(cr.hi, cr.hi), f2(cr.lo, cr.lo));
  const dfc2 b = dfc2_mulv(dfc2_swap(v), f2(-ci.hi, ci.hi), f2(-ci.lo, ci.lo));
  return dfc2_add(a, b);
}

__device__ __forceinline__ dfc2 dfc2_from_double2(double2 s) {
  const df r = df_from_double(s.x), i = df_from_double(s.y);
  return dfc2{f2(r.hi, i.hi), f2(r.lo, i.lo)};
}

__device__ __forceinline__ double2 dfc2_to_double2(dfc2 a) {
  return make_double2(df_to_double(df{a.hi.x, a.lo.x}), df_to_double(df{a.hi.y, a.lo.y}));
}

}  // namespace qs
