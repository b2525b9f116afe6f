// One-pass-per-gate kernels (state vectors and density matrices).
//
// Every kernel is a grid-stride loop over the selected indices with UNROLL
// independent iterations per thread in flight: all loads of an unrolled
// group are issued before any arithmetic, so each thread keeps
// UNROLL x (pair bytes) in flight.  Consecutive threads take consecutive
// indices, so each warp instruction touches contiguous memory whenever the
// fixed bits lie above the warp's span.
#pragma once
#include "common.cuh"
#include "pair_arith.cuh"

namespace qs {

// State-vector pass (Eq. 1): for the idx-th selected pair, j = deposit(idx)
// has the target bit 0 and every control bit 1; (a[j], a[j + stride]) <- G.
template <typename R, int K, int UNROLL>
__global__ void __launch_bounds__(256) k_sv_pair(cvec<R>* __restrict__ a, int64_t nsel,
                                                 int64_t stride, Fixed fx, Mat2<R> g) {
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; base < nsel;
       base += nthr * UNROLL) {
    int64_t j[UNROLL];
    cvec<R> x[UNROLL], y[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const int64_t idx = base + u * nthr;
      j[u] = idx < nsel ? deposit(idx, fx) : -1;
      if (j[u] >= 0) { x[u] = a[j[u]]; y[u] = a[j[u] + stride]; }
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      if (j[u] < 0) continue;
      pair_apply<R, K, false>(x[u], y[u], g);
      a[j[u]] = x[u];
      a[j[u] + stride] = y[u];
    }
  }
}

// Diagonal state-vector gates on the selected amplitudes (all fixed bits 1):
// PHASE multiplies by (c, s) = exp(i phi); SIGN negates (CZ, multi-controlled
// phase flip).
// DK_PHASE: times (c + i s); DK_SIGN: negate; DK_PHASEU: times (1 + i s), a
// phase whose real factor c the caller keeps (2 FMAs instead of 4 operations).
enum DiagKind { DK_PHASE = 0, DK_SIGN = 1, DK_PHASEU = 2 };

template <typename R, int K, int UNROLL>
__global__ void __launch_bounds__(256) k_sv_diag(cvec<R>* __restrict__ a, int64_t nsel,
                                                 Fixed fx, R c, R s) {
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; base < nsel;
       base += nthr * UNROLL) {
    int64_t j[UNROLL];
    cvec<R> x[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const int64_t idx = base + u * nthr;
      j[u] = idx < nsel ? deposit(idx, fx) : -1;
      if (j[u] >= 0) x[u] = a[j[u]];
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      if (j[u] < 0) continue;
      cvec<R> v = x[u];
      if constexpr (K == DK_SIGN) {
        v.x = neg_bits(v.x); v.y = neg_bits(v.y);
      } else if constexpr (K == DK_PHASEU) {
        v.x = fma(-s, x[u].y, x[u].x);
        v.y = fma(s, x[u].x, x[u].y);
      } else {
        v.x = c * x[u].x - s * x[u].y;
        v.y = s * x[u].x + c * x[u].y;
      }
      a[j[u]] = v;
    }
  }
}

// The same diagonal update on groups of V consecutive selected amplitudes
// (valid when every fixed bit is at position >= log2 V, so that deposit(g V)
// starts a run of V selected amplitudes): one index computation per V
// amplitudes and 16-byte vector accesses for complex64.
template <typename R, int K, int V, int UNROLL>
__global__ void __launch_bounds__(256) k_sv_diag_v(cvec<R>* __restrict__ a, int64_t ngroups,
                                                   Fixed fx, R c, R s) {
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; base < ngroups;
       base += nthr * UNROLL) {
    int64_t j[UNROLL];
    cvec<R> x[UNROLL][V];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const int64_t g = base + u * nthr;
      j[u] = g < ngroups ? deposit(g * V, fx) : -1;
      if (j[u] < 0) continue;
      if constexpr (sizeof(R) == 4 && V >= 2) {
#pragma unroll
        for (int w = 0; w < V; w += 2) {
          const float4 q = *reinterpret_cast<const float4*>(a + j[u] + w);
          x[u][w] = cvec<R>{q.x, q.y};
          x[u][w + 1] = cvec<R>{q.z, q.w};
        }
      } else {
#pragma unroll
        for (int w = 0; w < V; ++w) x[u][w] = a[j[u] + w];
      }
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      if (j[u] < 0) continue;
      cvec<R> v[V];
#pragma unroll
      for (int w = 0; w < V; ++w) {
        const cvec<R> y = x[u][w];
        if constexpr (K == DK_SIGN) {
          v[w].x = neg_bits(y.x); v[w].y = neg_bits(y.y);
        } else if constexpr (K == DK_PHASEU) {
          v[w].x = fma(-s, y.y, y.x);
          v[w].y = fma(s, y.x, y.y);
        } else {
          v[w].x = c * y.x - s * y.y;
          v[w].y = s * y.x + c * y.y;
        }
      }
      if constexpr (sizeof(R) == 4 && V >= 2) {
#pragma unroll
        for (int w = 0; w < V; w += 2)
          *reinterpret_cast<float4*>(a + j[u] + w) = make_float4(v[w].x, v[w].y, v[w + 1].x, v[w + 1].y);
      } else {
#pragma unroll
        for (int w = 0; w < V; ++w) a[j[u] + w] = v[w];
      }
    }
  }
}

// ---------------------------------------------------------- density matrix
// Quad pass of Eq. 2: for a quad base j (bits t and t+N zero) the four
// entries v[r][c] = a[j + r 2^t + c 2^(t+N)] (r = row bit, c = column bit).
// G acts on the row bit where the row controls hold (G_t), conj(G) on the
// column bit where the column controls hold (G*_{t+N}).
template <typename R, int K, int UNROLL>
__global__ void __launch_bounds__(256) k_dm_gate(cvec<R>* __restrict__ a, int64_t nsel,
                                                 int64_t rstride, int64_t cstride,
                                                 uint64_t rmask, uint64_t cmask, Fixed fx,
                                                 Mat2<R> g) {
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; base < nsel;
       base += nthr * UNROLL) {
    int64_t j[UNROLL];
    cvec<R> v[UNROLL][4];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const int64_t idx = base + u * nthr;
      j[u] = idx < nsel ? deposit(idx, fx) : -1;
      if (j[u] >= 0) {
        v[u][0] = a[j[u]];
        v[u][1] = a[j[u] + rstride];
        v[u][2] = a[j[u] + cstride];
        v[u][3] = a[j[u] + rstride + cstride];
      }
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      if (j[u] < 0) continue;
      const uint64_t jj = uint64_t(j[u]);
      if ((jj & rmask) == rmask) {
        pair_apply<R, K, false>(v[u][0], v[u][1], g);
        pair_apply<R, K, false>(v[u][2], v[u][3], g);
      }
      if ((jj & cmask) == cmask) {
        pair_apply<R, K, true>(v[u][0], v[u][2], g);
        pair_apply<R, K, true>(v[u][1], v[u][3], g);
      }
      a[j[u]] = v[u][0];
      a[j[u] + rstride] = v[u][1];
      a[j[u] + cstride] = v[u][2];
      a[j[u] + rstride + cstride] = v[u][3];
    }
  }
}

// Depolarising channel on the (row t, column t) block of every quad:
// diagonal entries d0' = (1 - 2p/3) d0 + (2p/3) d1 (and symmetrically),
// off-diagonal entries scaled by (1 - 4p/3).  Arguments: keep = 1 - 2p/3,
// move = 2p/3, off = 1 - 4p/3.
template <typename R, int UNROLL>
__global__ void __launch_bounds__(256) k_dm_depol(cvec<R>* __restrict__ a, int64_t nsel,
                                                  int64_t rstride, int64_t cstride, Fixed fx,
                                                  R keep, R move, R off) {
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; base < nsel;
       base += nthr * UNROLL) {
    int64_t j[UNROLL];
    cvec<R> v[UNROLL][4];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      const int64_t idx = base + u * nthr;
      j[u] = idx < nsel ? deposit(idx, fx) : -1;
      if (j[u] >= 0) {
        v[u][0] = a[j[u]];
        v[u][1] = a[j[u] + rstride];
        v[u][2] = a[j[u] + cstride];
        v[u][3] = a[j[u] + rstride + cstride];
      }
    }
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
      if (j[u] < 0) continue;
      const cvec<R> d0 = v[u][0], d1 = v[u][3];
      cvec<R> o0 = v[u][1], o1 = v[u][2];
      cvec<R> n0, n1;
      n0.x = keep * d0.x + move * d1.x; n0.y = keep * d0.y + move * d1.y;
      n1.x = keep * d1.x + move * d0.x; n1.y = keep * d1.y + move * d0.y;
      o0.x *= off; o0.y *= off; o1.x *= off; o1.y *= off;
      a[j[u]] = n0;
      a[j[u] + rstride] = o0;
      a[j[u] + cstride] = o1;
      a[j[u] + rstride + cstride] = n1;
    }
  }
}

// Density-matrix diagonal operations, one predicate per entry n = j + 2^N k:
//  DM_SIGN:    P rho P with P = sign flip where all bits of `mask` are set:
//              entry negated when exactly one of (row bits, column bits) has
//              every mask bit set.
//  DM_PHASE:   diag(1, e^{i phi}) on qubit t with controls: row factor
//              e^{i phi} where row bit t and row controls are 1, column
//              factor e^{-i phi} likewise; product applied.
//  DM_DEPHASE: entries with row bit t != column bit t scaled by f = 1 - 2p.
// Entries left unchanged are neither read nor written.
enum DmDiagKind { DD_SIGN = 0, DD_PHASE = 1, DD_DEPHASE = 2 };

template <typename R, int K>
__global__ void __launch_bounds__(256) k_dm_diag(cvec<R>* __restrict__ a, int64_t dim, int N,
                                                 uint64_t mask, int t, R c, R s) {
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  const uint64_t cmask = mask << N;
  for (int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; n < dim; n += nthr) {
    const uint64_t un = uint64_t(n);
    if constexpr (K == DD_SIGN) {
      const bool r = (un & mask) == mask, k = (un & cmask) == cmask;
      if (r != k) {
        cvec<R> v = a[n];
        v.x = neg_bits(v.x); v.y = neg_bits(v.y);
        a[n] = v;
      }
    } else if constexpr (K == DD_PHASE) {
      const bool r = ((un >> t) & 1) && (un & mask) == mask;
      const bool k = ((un >> (t + N)) & 1) && (un & cmask) == cmask;
      if (r != k) {
        const R ss = r ? s : -s;  // e^{i phi} (row only) or e^{-i phi} (column only)
        cvec<R> v = a[n], w;
        w.x = c * v.x - ss * v.y;
        w.y = ss * v.x + c * v.y;
        a[n] = w;
      }
    } else {
      if (((un >> t) & 1) != ((un >> (t + N)) & 1)) {
        cvec<R> v = a[n];
        v.x *= c; v.y *= c;
        a[n] = v;
      }
    }
  }
}

// ------------------------------------------------------------- utilities
template <typename R>
__global__ void k_fill(cvec<R>* __restrict__ a, int64_t count, R re, R im) {
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  for (int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; n < count; n += nthr) {
    cvec<R> v; v.x = re; v.y = im;
    a[n] = v;
  }
}

// a <- a (re + i im): applies a register's pending scalar factor.
template <typename R>
__global__ void k_scale(cvec<R>* __restrict__ a, int64_t count, R re, R im) {
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  for (int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; n < count; n += nthr) {
    const cvec<R> v = a[n];
    cvec<R> w;
    w.x = re * v.x - im * v.y;
    w.y = im * v.x + re * v.y;
    a[n] = w;
  }
}

__global__ void k_f2d(const float2* __restrict__ s, double2* __restrict__ d, int64_t count);
__global__ void k_d2f(const double2* __restrict__ s, float2* __restrict__ d, int64_t count);

}  // namespace qs
