// Shared device definitions of the simulator kernels.
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#include <cuda_runtime.h>
#endif

namespace qs {

template <typename R> struct cplx_of;
template <> struct cplx_of<double> { using type = double2; };
template <> struct cplx_of<float> { using type = float2; };
template <typename R> using cvec = typename cplx_of<R>::type;

// 2x2 complex matrix, row-major: [0]=m00 [1]=m01 [2]=m10 [3]=m11.
template <typename R> struct Mat2 { R re[4], im[4]; };

// Positions of index bits held fixed while a kernel enumerates the other
// bits: pos[] ascending, value of pos[k] in bit k of `vals`.
constexpr int kMaxFixed = 64;
struct Fixed {
  int n;
  uint64_t vals;
  uint8_t pos[kMaxFixed];
};

// The idx-th index (in increasing order) whose bits at s.pos[] equal
// s.vals: the other bits of the result are the bits of idx, in order.
// With one fixed bit q of value 0 this is n_i of Eq. 1.
__device__ __forceinline__ int64_t deposit(int64_t idx, const Fixed& s) {
#pragma unroll 1
  for (int k = 0; k < s.n; ++k) {
    const int p = s.pos[k];
    const int64_t low = idx & ((int64_t(1) << p) - 1);
    idx = ((idx >> p) << (p + 1)) | low | (int64_t((s.vals >> k) & 1) << p);
  }
  return idx;
}

// Negation by flipping the IEEE sign bit (integer op, no FP pipe).
__device__ __forceinline__ double neg_bits(double x) {
  return __hiloint2double(__double2hiint(x) ^ 0x80000000, __double2loint(x));
}
__device__ __forceinline__ float neg_bits(float x) {
  return __int_as_float(__float_as_int(x) ^ 0x80000000);
}

// float -> double, exactly, without the FP64 pipe: the double has the
// float's sign, its exponent rebiased by 1023 - 127 = 896 and its 23-bit
// significand followed by 29 zero bits (IEEE 754 binary32 / binary64
// layouts).  A subnormal is first scaled by 2^64 on the FP32 pipe (exact:
// a power of two, into the normal range) and its exponent lowered by 64;
// zero keeps exponent 0, infinities and NaN take 2047 with their
// significand bits.  Selects, not branches: on B300 a conversion
// instruction, even predicated off, occupies the FP64 pipe that the FMAs of
// the FP64 reductions need (2 conversions and 2 FMAs per complex64
// amplitude).  The value is the conversion's, so results do not change.
__device__ __forceinline__ double widen(float x) {
  const uint32_t f0 = __float_as_uint(x);
  const bool sub = (f0 & 0x7F800000u) == 0u && (f0 & 0x007FFFFFu) != 0u;
  const uint32_t f = __float_as_uint(sub ? x * 18446744073709551616.0f : x);  // x 2^64
  const uint32_t e = (f >> 23) & 0xFFu, m = f & 0x007FFFFFu;
  const uint32_t ed = e == 0u ? 0u : (e == 0xFFu ? 0x7FFu : e + 896u - (sub ? 64u : 0u));
  return __hiloint2double(int((f & 0x80000000u) | (ed << 20) | (m >> 3)), int(m << 29));
}
__device__ __forceinline__ double widen(double x) { return x; }

}  // namespace qs
