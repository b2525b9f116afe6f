// Multi-target gates: a dense 2^M x 2^M unitary on M target qubits (Eq. 1
// with the amplitude pair replaced by a block of 2^M amplitudes; the paper
// notes the density-matrix rule holds for multi-qubit gates, Sec. II.B.1).
#pragma once
#include "common.cuh"

namespace qs {

constexpr int kMaxMultiTargets = 5;

template <typename R, int M>
struct MultiParams {
  uint8_t t[8];                     // target qubits; bit k of the block index is t[k]
  cvec<R> u[1 << (2 * M)];          // row-major matrix
};

// One block per selected base index j = deposit(idx) (target bits 0, control
// bits 1): gather the 2^M amplitudes, multiply by the matrix, scatter.
template <typename R, int M>
__global__ void __launch_bounds__(256) k_sv_multi(cvec<R>* __restrict__ a, int64_t nsel, Fixed fx,
                                                  const __grid_constant__ MultiParams<R, M> p) {
  constexpr int B = 1 << M;
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  auto off = [&](int l) {
    int64_t o = 0;
#pragma unroll
    for (int k = 0; k < M; ++k)
      if ((l >> k) & 1) o += int64_t(1) << p.t[k];
    return o;
  };
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < nsel; idx += nthr) {
    const int64_t j = deposit(idx, fx);
    cvec<R> v[B];
#pragma unroll
    for (int l = 0; l < B; ++l) v[l] = a[j + off(l)];
#pragma unroll
    for (int r = 0; r < B; ++r) {
      // four FMA chains per row (written out: `re += gx vx - gy vy` would
      // round the second product separately and cost a multiply, an FMA and
      // an add for every two products)
      R re = R(0), im = R(0);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const cvec<R> g = p.u[r * B + c];
        re = fma(g.x, v[c].x, re);
        re = fma(-g.y, v[c].y, re);
        im = fma(g.x, v[c].y, im);
        im = fma(g.y, v[c].x, im);
      }
      cvec<R> w;
      w.x = re;
      w.y = im;
      a[j + off(r)] = w;
    }
  }
}

// Complex64 matrix entries duplicated for paired FP32 arithmetic: u[e] =
// (re, re, im, im) of entry e.
template <int M>
struct MultiParamsF2 {
  uint8_t t[8];
  float4 u[1 << (2 * M)];
};

// k_sv_multi for complex64 with paired FP32 FMAs (`fma.rn.f32x2`): per row,
// P = sum_c Re(g_c) (x_c, y_c) and Q = sum_c Im(g_c) (x_c, y_c), both on the
// amplitude pair as stored, then Re = P.x - Q.y and Im = P.y + Q.x: two
// paired FMAs per complex multiply-add and no operand swap.
template <int M>
__global__ void __launch_bounds__(256) k_sv_multi_f2(float2* __restrict__ a, int64_t nsel, Fixed fx,
                                                     const __grid_constant__ MultiParamsF2<M> p) {
  constexpr int B = 1 << M;
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  auto off = [&](int l) {
    int64_t o = 0;
#pragma unroll
    for (int k = 0; k < M; ++k)
      if ((l >> k) & 1) o += int64_t(1) << p.t[k];
    return o;
  };
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < nsel; idx += nthr) {
    const int64_t j = deposit(idx, fx);
    float2 v[B];
#pragma unroll
    for (int l = 0; l < B; ++l) v[l] = a[j + off(l)];
#pragma unroll
    for (int r = 0; r < B; ++r) {
      float2 P = make_float2(0.f, 0.f), Q = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const float4 g = p.u[r * B + c];
        P = __ffma2_rn(make_float2(g.x, g.y), v[c], P);
        Q = __ffma2_rn(make_float2(g.z, g.w), v[c], Q);
      }
      a[j + off(r)] = make_float2(P.x - Q.y, P.y + Q.x);
    }
  }
}

}  // namespace qs
