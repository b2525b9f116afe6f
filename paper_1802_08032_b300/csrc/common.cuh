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

}  // namespace qs
