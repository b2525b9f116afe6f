// FP64 reductions (total probability, outcome probability, trace, purity)
// and measurement collapse.
//
// Two stages with a fixed grid: each CTA sums its grid-strided share in
// FP64 in a fixed order and writes one partial; one CTA then sums the
// partials in a fixed order.  The result is therefore the same bit for bit
// from run to run on a given GPU (c64 inputs are widened to FP64 first).
#pragma once
#include "common.cuh"

namespace qs {

constexpr int kRedThreads = 512;

constexpr int kRedMaxBlocks = 1184;  // 148 SMs x 8

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;  // valid in thread 0
}

// sum over selected indices j = deposit(idx) of |a_j|^2.
template <typename R, int UNROLL>
__global__ void __launch_bounds__(kRedThreads) k_sumsq(const cvec<R>* __restrict__ a,
                                                       int64_t nsel, Fixed fx,
                                                       double* __restrict__ partial) {
  __shared__ double sh[32];
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  double acc = 0.0;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; base < nsel;
       base += nthr * UNROLL) {
    cvec<R> x[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const int64_t idx = base + u * nthr;
      if (idx < nsel) x[u] = a[deposit(idx, fx)];
      else { x[u].x = R(0); x[u].y = R(0); }
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const double re = widen(x[u].x), im = widen(x[u].y);
      acc = fma(re, re, acc);
      acc = fma(im, im, acc);
    }
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Density matrix: sum over rows j (optionally only those with bit q = o) of
// Re rho[j][j], stored at j + 2^N j.
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_sumdiag(const cvec<R>* __restrict__ a, int N,
                                                         int q, int o,
                                                         double* __restrict__ partial) {
  __shared__ double sh[32];
  const int64_t d = int64_t(1) << N;
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  double acc = 0.0;
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < d; j += nthr) {
    if (q < 0 || ((j >> q) & 1) == o) acc += double(a[j + (j << N)].x);
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// sum over j of conj(a_j) b_j in FP64 (a and b of either precision, widened
// first): partial[blockIdx.x] = real part, partial[gridDim.x + blockIdx.x] =
// imaginary part.
template <typename RA, typename RB, int UNROLL>
__global__ void __launch_bounds__(kRedThreads) k_inner(const cvec<RA>* __restrict__ a,
                                                       const cvec<RB>* __restrict__ b, int64_t n,
                                                       double* __restrict__ partial) {
  __shared__ double sh[32];
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  double re = 0.0, im = 0.0;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; base < n; base += nthr * UNROLL) {
    cvec<RA> x[UNROLL];
    cvec<RB> y[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const int64_t j = base + u * nthr;
      if (j < n) {
        x[u] = a[j];
        y[u] = b[j];
      } else {
        x[u].x = RA(0); x[u].y = RA(0);
        y[u].x = RB(0); y[u].y = RB(0);
      }
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const double ar = widen(x[u].x), ai = widen(x[u].y), br = widen(y[u].x), bi = widen(y[u].y);
      re = fma(ar, br, re);
      re = fma(ai, bi, re);
      im = fma(ar, bi, im);
      im = fma(-ai, br, im);
    }
  }
  const double sr = block_sum(re, sh);
  __syncthreads();
  const double si = block_sum(im, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = sr;
    partial[gridDim.x + blockIdx.x] = si;
  }
}

// Second stage: out[0] = sum of partial[0..n) in a fixed order.
__global__ void __launch_bounds__(1024) k_sum_partials(const double* __restrict__ partial, int n,
                                                       double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) out[0] = s;
}

// Collapse of a state vector onto bit q = o: a_j <- a_j * scale (FP64) where
// bit q = o, else 0.  Entries set to zero are not read.
template <typename R>
__global__ void __launch_bounds__(256) k_collapse_sv(cvec<R>* __restrict__ a, int64_t dim, int q,
                                                     int o, double scale) {
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  for (int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; n < dim; n += nthr) {
    cvec<R> v;
    if (((n >> q) & 1) == o) {
      v = a[n];
      v.x = R(double(v.x) * scale);
      v.y = R(double(v.y) * scale);
    } else {
      v.x = R(0); v.y = R(0);
    }
    a[n] = v;
  }
}

// Collapse of a density matrix: keep entries whose row bit q and column bit
// q both equal o, times scale = 1/p; zero elsewhere.
template <typename R>
__global__ void __launch_bounds__(256) k_collapse_dm(cvec<R>* __restrict__ a, int64_t dim, int N,
                                                     int q, int o, double scale) {
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  for (int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; n < dim; n += nthr) {
    cvec<R> v;
    if (((n >> q) & 1) == o && ((n >> (q + N)) & 1) == o) {
      v = a[n];
      v.x = R(double(v.x) * scale);
      v.y = R(double(v.y) * scale);
    } else {
      v.x = R(0); v.y = R(0);
    }
    a[n] = v;
  }
}

}  // namespace qs
