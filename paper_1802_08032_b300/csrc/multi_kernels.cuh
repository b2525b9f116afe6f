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
      R re = R(0), im = R(0);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const cvec<R> g = p.u[r * B + c];
        re += g.x * v[c].x - g.y * v[c].y;
        im += g.x * v[c].y + g.y * v[c].x;
      }
      cvec<R> w;
      w.x = re;
      w.y = im;
      a[j + off(r)] = w;
    }
  }
}

}  // namespace qs
