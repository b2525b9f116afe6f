// Multi-target gates: a dense 2^M x 2^M unitary on M target qubits (Eq. 1
// with the amplitude pair replaced by a block of 2^M amplitudes; the paper
// notes the density-matrix rule holds for multi-qubit gates, Sec. II.B.1).
#pragma once
#include "common.cuh"
#include "dfloat.cuh"

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

// Tables of k_sv_multi_f2_tile.  A tile is every combination of the M
// targets and the 8 lowest free qubits (neither target nor control): local
// index bit k is qubit lpos[k] (ascending), so the lowest local bits are the
// lowest qubits and a warp's 32 consecutive local indices are (without
// controls among qubits 0..4) 32 consecutive amplitudes.  Shared-memory slot
// of local index x: x ^ sw(x), sw XOR-linear with sw(bit k) = swz[k] (bits
// 0..3 unchanged), chosen so that the 16 blocks a half-warp works on fall in
// 16 different bank pairs; both access patterns then split into per-thread
// and per-element parts (the bits are disjoint, so OR = XOR).
template <int M>
struct MultiTileParams {
  float4 u[1 << (2 * M)];      // matrix entries duplicated (re, re, im, im)
  int64_t goff_hi[1 << M];     // global offset of local index 256 i
  uint16_t sm_hi[1 << M];      // slot part of local index 256 i
  uint16_t sm_l[1 << M];       // slot part of block element l (the target bits)
  uint8_t lpos[16];            // qubit of local bit k, k < M + 8
  uint8_t fpos[8];             // local bit of block-index bit j (the free local bits)
  uint8_t swz[16];             // swizzle of local bit k
};

// k_sv_multi_f2 for a target among the lowest qubits, where one thread's
// block is a few short runs of contiguous amplitudes and per-block loads do
// not coalesce: a CTA loads a tile in address order into shared memory
// (2^M coalesced accesses a thread), each thread updates one block there
// (256 blocks a tile), and the tile is stored in address order.
template <int M>
__global__ void __launch_bounds__(256, M >= 4 ? 2 : 4) k_sv_multi_f2_tile(float2* __restrict__ a, int64_t ntiles, Fixed fx,
                                                          const __grid_constant__ MultiTileParams<M> p) {
  constexpr int B = 1 << M;
  __shared__ float2 tile[256 * B];
  const uint32_t t = threadIdx.x;
  int64_t goff_t = 0;
  uint32_t sm_t = t, lam_b = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if ((t >> k) & 1u) {
      goff_t += int64_t(1) << p.lpos[k];
      sm_t ^= p.swz[k];
      lam_b |= 1u << p.fpos[k];
    }
  uint32_t sm_b = lam_b;
#pragma unroll
  for (int k = 0; k < M + 8; ++k)
    if ((lam_b >> k) & 1u) sm_b ^= p.swz[k];
  int64_t tau = blockIdx.x;
  if (tau >= ntiles) return;
  int64_t base = deposit(tau, fx) + goff_t;
  float2 x[B];
#pragma unroll
  for (int i = 0; i < B; ++i) x[i] = a[base + p.goff_hi[i]];
  for (;;) {
#pragma unroll
    for (int i = 0; i < B; ++i) tile[sm_t ^ p.sm_hi[i]] = x[i];
    __syncthreads();
    // the next tile's loads go out before this tile's arithmetic and stores
    // (the condition is uniform over the CTA)
    const int64_t tau_n = tau + gridDim.x;
    int64_t base_n = 0;
    if (tau_n < ntiles) {
      base_n = deposit(tau_n, fx) + goff_t;
#pragma unroll
      for (int i = 0; i < B; ++i) x[i] = a[base_n + p.goff_hi[i]];
    }
    float2 v[B];
#pragma unroll
    for (int l = 0; l < B; ++l) v[l] = tile[sm_b ^ p.sm_l[l]];
#pragma unroll
    for (int r = 0; r < B; ++r) {
      float2 P = make_float2(0.f, 0.f), Q = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const float4 g = p.u[r * B + c];
        P = __ffma2_rn(make_float2(g.x, g.y), v[c], P);
        Q = __ffma2_rn(make_float2(g.z, g.w), v[c], Q);
      }
      tile[sm_b ^ p.sm_l[r]] = make_float2(P.x - Q.y, P.y + Q.x);  // this thread's own slots
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < B; ++i) a[base + p.goff_hi[i]] = tile[sm_t ^ p.sm_hi[i]];
    if (tau_n >= ntiles) break;
    __syncthreads();  // the next tile reuses the buffer
    tau = tau_n;
    base = base_n;
  }
}

// Complex128 matrix entries as double-float pairs: u[e] = (Re hi, Re lo,
// Im hi, Im lo) of entry e.
template <int M>
struct MultiParamsDF {
  uint8_t t[8];
  float4 u[1 << (2 * M)];
};

// k_sv_multi for complex128 amplitudes in double-float arithmetic on the
// FP32 pipes (env option "arith" 1).  Each amplitude is split into a
// packed pair hi = (Re hi, Im hi), lo = (Re lo, Im lo); per row, P = sum_c
// Re(g_c) v_c and Q = sum_c Im(g_c) v_c as in k_sv_multi_f2, each product
// formed exactly (p = g_hi v_hi, its rounding error by an FMA, plus the two
// cross terms g_hi v_lo + g_lo v_hi), the high parts summed by error-free
// two-sums and every low part accumulated in float; then (P.x - Q.y,
// P.y + Q.x) by one double-float addition.  Error: about 2^M units of 2^-48
// of the block's norm per gate (the low-part sum), far below 1e-12.
template <int M>
__global__ void __launch_bounds__(256) k_sv_multi_df(double2* __restrict__ a, int64_t nsel, Fixed fx,
                                                     const __grid_constant__ MultiParamsDF<M> p) {
  constexpr int B = 1 << M;
  const int64_t nthr = int64_t(gridDim.x) * blockDim.x;
  auto off = [&](int l) {
    int64_t o = 0;
#pragma unroll
    for (int k = 0; k < M; ++k)
      if ((l >> k) & 1) o += int64_t(1) << p.t[k];
    return o;
  };
  // accumulates g v (g a real double-float, broadcast to both halves) into
  // the high sum S and the low sum E
  auto mac = [](float2& S, float2& E, const dfc2& v, float gh, float gl, bool first) {
    const float2 G = f2(gh, gh);
    const float2 p = mul2(v.hi, G);
    const float2 np = mul2(v.hi, f2(-gh, -gh));  // -p exactly
    float2 e = fma2(v.hi, G, np);
    e = fma2(v.hi, f2(gl, gl), e);
    e = fma2(v.lo, G, e);
    if (first) {
      S = p;
      E = e;
    } else {
      const dfc2 t = two_sum2(S, p);
      S = t.hi;
      E = add2(E, add2(t.lo, e));
    }
  };
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < nsel; idx += nthr) {
    const int64_t j = deposit(idx, fx);
    dfc2 v[B];
#pragma unroll
    for (int l = 0; l < B; ++l) v[l] = dfc2_from_double2(a[j + off(l)]);
#pragma unroll
    for (int r = 0; r < B; ++r) {
      float2 Ps, Pe, Qs, Qe;
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const float4 g = p.u[r * B + c];
        mac(Ps, Pe, v[c], g.x, g.y, c == 0);
        mac(Qs, Qe, v[c], g.z, g.w, c == 0);
      }
      const dfc2 P = fast_two_sum2(Ps, Pe), Q = fast_two_sum2(Qs, Qe);
      const dfc2 iQ{f2(-Q.hi.y, Q.hi.x), f2(-Q.lo.y, Q.lo.x)};  // i Q
      a[j + off(r)] = dfc2_to_double2(dfc2_add(P, iQ));
    }
  }
}

}  // namespace qs
