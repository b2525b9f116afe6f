// Arithmetic of the fused tile engine: the operations a thread applies to
// its 2^R register amplitudes (pair updates on a register bit, phases, sign
// flips, channel mixes), in FP32, FP64 or double-float.  Shared by the
// interpreting fused kernel (fused_kernel.cuh) and the pass kernels
// compiled at run time for one pass's operation list (jit.cpp), so both
// apply bit-for-bit the same arithmetic; compiles under NVRTC as well as
// nvcc.
#pragma once
#include "common.cuh"
#include "dfloat.cuh"
#include "fused_types.h"
#include "pair_arith.cuh"

namespace qs {

// ------------------------------------------------------------- arithmetic
// Plain arithmetic on the storage type (complex64: FP32, complex128: FP64).
template <typename R>
struct PlainArith {
  using Store = cvec<R>;
  using Cplx = cvec<R>;
  __device__ static R cf(const FOp& op, int e) {
    if constexpr (sizeof(R) == 8) return op.c.d[e];
    else return op.c.f[e];
  }
  __device__ static Cplx from_store(const Store& s) { return s; }
  __device__ static Store to_store(const Cplx& c) { return c; }
  // FP64 only: unscaled H / sqrt(X) / sqrt(Y) with a real factor on either
  // input (see pair_side_on_bit)
  static constexpr bool kSide = sizeof(R) == 8;
  // The unscaled butterfly of K applied to (f x, y): one FMA per output
  // component, f = c0.
  template <int K, bool CONJ>
  __device__ static void pair_xs(Cplx& x, Cplx& y, const FOp& op) {
    const R f = cf(op, 0);
    const Cplx u = x;
    if constexpr (K == PK_H) {  // (f x + y, f x - y)
      x.x = fma(f, u.x, y.x); x.y = fma(f, u.y, y.y);
      y.x = fma(f, u.x, -y.x); y.y = fma(f, u.y, -y.y);
    } else if constexpr (K == PK_SX && !CONJ) {  // (f x - i y, -i f x + y)
      x.x = fma(f, u.x, y.y); x.y = fma(f, u.y, -y.x);
      y.x = fma(f, u.y, y.x); y.y = fma(-f, u.x, y.y);
    } else if constexpr (K == PK_SX) {  // (f x + i y, i f x + y)
      x.x = fma(f, u.x, -y.y); x.y = fma(f, u.y, y.x);
      y.x = fma(-f, u.y, y.x); y.y = fma(f, u.x, y.y);
    } else {  // sqrt(Y): (f x - y, f x + y)
      x.x = fma(f, u.x, -y.x); x.y = fma(f, u.y, -y.y);
      y.x = fma(f, u.x, y.x); y.y = fma(f, u.y, y.y);
    }
  }
  template <int K, bool CONJ>
  __device__ static void pair_t(Cplx& x, Cplx& y, const FOp& op) {
    if constexpr (K == PK_GEN) {
      Mat2<R> g;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        g.re[e] = cf(op, 2 * e);
        g.im[e] = cf(op, 2 * e + 1);
      }
      pair_apply<R, K, CONJ>(x, y, g);
    } else if constexpr (sizeof(R) == 4 && (K == PK_H || K == PK_SX || K == PK_SY)) {
      // FP32: each real butterfly (a, b) -> (a + c b, c b - a) or
      // (a - c b, a + c b), c = the y factor c0, is computed in place, the
      // second output from the first by one FMA with the factor 2c
      // (c b - a = 2c b - (a + c b)).  Both outputs then stay in the inputs'
      // registers, which saves a register move per output; the second output
      // carries one extra rounding of |a + c b|.
      const R c = cf(op, 0), c2 = 2.f * c;
      // real matrices: one paired FMA covers the real and imaginary parts
      // (each half rounds as the scalar FMA would)
      if constexpr (K == PK_H) {  // unscaled: (x + c y, x - c y)
        x = __ffma2_rn(make_float2(c, c), y, x);
        y = __ffma2_rn(y, make_float2(-c2, -c2), x);
      } else if constexpr (K == PK_SY) {  // [[1, -1], [1, 1]]: (x - c y, x + c y)
        x = __ffma2_rn(make_float2(-c, -c), y, x);
        y = __ffma2_rn(y, make_float2(c2, c2), x);
      } else if constexpr (!CONJ) {  // [[1, -i], [-i, 1]]
        x.x = fmaf(c, y.y, x.x); y.y = fmaf(y.y, c2, -x.x);    // c y.im - x.re
        x.y = fmaf(-c, y.x, x.y); y.x = fmaf(y.x, c2, x.y);    // c y.re + x.im
      } else {  // [[1, i], [i, 1]]
        x.x = fmaf(-c, y.y, x.x); y.y = fmaf(y.y, c2, x.x);    // c y.im + x.re
        x.y = fmaf(c, y.x, x.y); y.x = fmaf(y.x, c2, -x.y);    // c y.re - x.im
      }
    } else if constexpr (K == PK_H) {  // unscaled: (x + c y, x - c y); FMA with c = 1 is the add
      const R c = cf(op, 0);
      const Cplx u = x;
      x.x = fma(c, y.x, u.x); x.y = fma(c, y.y, u.y);
      y.x = fma(-c, y.x, u.x); y.y = fma(-c, y.y, u.y);
    } else if constexpr (K == PK_SX) {  // [[1, -i], [-i, 1]]  (conj: [[1, i], [i, 1]])
      const R c = cf(op, 0);
      const Cplx u = x;
      if constexpr (!CONJ) {
        x.x = fma(c, y.y, u.x); x.y = fma(-c, y.x, u.y); y.x = fma(c, y.x, u.y); y.y = fma(c, y.y, -u.x);
      } else {
        x.x = fma(-c, y.y, u.x); x.y = fma(c, y.x, u.y); y.x = fma(c, y.x, -u.y); y.y = fma(c, y.y, u.x);
      }
    } else if constexpr (K == PK_SY) {  // [[1, -1], [1, 1]] (real)
      const R c = cf(op, 0);
      const Cplx u = x;
      x.x = fma(-c, y.x, u.x); x.y = fma(-c, y.y, u.y);
      y.x = fma(c, y.x, u.x); y.y = fma(c, y.y, u.y);
    } else if constexpr (K == PK_X) {
      const Cplx t = x;
      x = y;
      y = t;
    }
  }
  __device__ static Cplx phase(const Cplx& v, const FOp& op) {
    const R c = cf(op, 0), s = cf(op, 1);
    Cplx w;
    // explicit FMAs: the same rounding wherever this is compiled (the
    // interpreting kernel and the runtime-compiled ones)
    w.x = fma(c, v.x, -(s * v.y));
    w.y = fma(s, v.x, c * v.y);
    return w;
  }
  // FP64: flip the sign bits (integer pipe; the FP64 pipe is the bottleneck).
  // FP32: multiply by -1 (exact; the FMA pipe instead of the busier integer
  // pipe), one paired multiply for both parts.
  __device__ static Cplx negate(const Cplx& v) {
    Cplx w;
    if constexpr (sizeof(R) == 4) {
      w = __fmul2_rn(v, make_float2(-1.f, -1.f));
    } else {
      w.x = neg_bits(v.x);
      w.y = neg_bits(v.y);
    }
    return w;
  }
  // (1 + i t) v, t = c[E]: the unscaled phase
  template <int E = 0>
  __device__ static Cplx phase_u(const Cplx& v, const FOp& op) {
    const R t = cf(op, E);
    Cplx w;
    w.x = fma(-t, v.y, v.x);
    w.y = fma(t, v.x, v.y);
    return w;
  }
  // Shear along a register bit: MODE 0 (x - t y, y + t' x), MODE 1
  // (t x - y, x + t y), t = c0, t' = c4.
  template <int MODE>
  __device__ static void shear(Cplx& x, Cplx& y, const FOp& op) {
    const R t = cf(op, 0);
    const Cplx u = x;
    if constexpr (MODE == 0) {
      const R t2 = cf(op, 4);
      x.x = fma(-t, y.x, u.x);
      x.y = fma(-t, y.y, u.y);
      y.x = fma(t2, u.x, y.x);
      y.y = fma(t2, u.y, y.y);
    } else {
      x.x = fma(t, u.x, -y.x);
      x.y = fma(t, u.y, -y.y);
      y.x = fma(t, y.x, u.x);
      y.y = fma(t, y.y, u.y);
    }
  }
  // i v: a swap and a sign flip, no arithmetic
  __device__ static Cplx mul_i(const Cplx& v) {
    Cplx w;
    w.x = neg_bits(v.y);
    w.y = v.x;
    return w;
  }

  __device__ static Cplx scale(const Cplx& v, const FOp& op, int e) {
    const R f = cf(op, e);
    Cplx w;
    w.x = v.x * f;
    w.y = v.y * f;
    return w;
  }
  // Depolarising mix of the diagonal pair (x, y) = (rho_00, rho_11) up to
  // the deferred factor 1 - m: (x + r y, y + r x), r = c0, one FMA per
  // component.
  __device__ static void depol_mix(Cplx& x, Cplx& y, const FOp& op) {
    const R r = cf(op, 0);
    const Cplx u = x;
    x.x = fma(r, y.x, u.x);
    x.y = fma(r, y.y, u.y);
    y.x = fma(r, u.x, y.x);
    y.y = fma(r, u.y, y.y);
  }
};

// Double-float arithmetic for complex128 storage: each real part is an
// unevaluated sum hi + lo of two floats (dfloat.cuh), held packed as
// hi = (re.hi, im.hi), lo = (re.lo, im.lo) so that the real and imaginary
// parts go through the paired FP32 instructions together.
struct DFArith {
  using Store = double2;
  using Cplx = dfc2;
  __device__ static df cf(const FOp& op, int e) { return df{op.c.f[e], op.c.f[8 + e]}; }
  static constexpr bool kSide = false;
  __device__ static Cplx from_store(const Store& s) { return dfc2_from_double2(s); }
  __device__ static Store to_store(const Cplx& c) { return dfc2_to_double2(c); }
  // multiply by -i: (re, im) -> (im, -re);  by +i: (re, im) -> (-im, re)
  __device__ static dfc2 mul_minus_i(const dfc2& a) {
    return dfc2{f2(a.hi.y, -a.hi.x), f2(a.lo.y, -a.lo.x)};
  }
  __device__ static dfc2 mul_plus_i(const dfc2& a) {
    return dfc2{f2(-a.hi.y, a.hi.x), f2(-a.lo.y, a.lo.x)};
  }
  template <int K, bool CONJ>
  __device__ static void pair_t(Cplx& x, Cplx& y, const FOp& op) {
    if constexpr (K == PK_GEN) {
      df g[4][2];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        g[e][0] = cf(op, 2 * e);
        g[e][1] = CONJ ? df_neg(cf(op, 2 * e + 1)) : cf(op, 2 * e + 1);
      }
      const dfc2 nx = dfc2_add(dfc2_cmul(x, g[0][0], g[0][1]), dfc2_cmul(y, g[1][0], g[1][1]));
      const dfc2 ny = dfc2_add(dfc2_cmul(x, g[2][0], g[2][1]), dfc2_cmul(y, g[3][0], g[3][1]));
      x = nx;
      y = ny;
    } else if constexpr (K == PK_H) {  // unscaled
      const dfc2 u = dfc2_add(x, y), v = dfc2_sub(x, y);
      x = u;
      y = v;
    } else if constexpr (K == PK_SX) {  // [[1, -i], [-i, 1]]  (conj: [[1, i], [i, 1]])
      const dfc2 u = x;
      if constexpr (!CONJ) {
        x = dfc2_add(u, mul_minus_i(y));
        y = dfc2_add(y, mul_minus_i(u));
      } else {
        x = dfc2_add(u, mul_plus_i(y));
        y = dfc2_add(y, mul_plus_i(u));
      }
    } else if constexpr (K == PK_SY) {  // [[1, -1], [1, 1]]
      const dfc2 u = x;
      x = dfc2_sub(u, y);
      y = dfc2_add(u, y);
    } else if constexpr (K == PK_X) {
      const dfc2 t = x;
      x = y;
      y = t;
    }
  }
  __device__ static Cplx phase(const Cplx& v, const FOp& op) { return dfc2_cmul(v, cf(op, 0), cf(op, 1)); }
  __device__ static Cplx mul_i(const Cplx& v) { return mul_plus_i(v); }
  template <int E = 0>
  __device__ static Cplx phase_u(const Cplx& v, const FOp& op) {
    return dfc2_cmul(v, df{1.f, 0.f}, cf(op, E));
  }
  template <int MODE>
  __device__ static void shear(Cplx& x, Cplx& y, const FOp& op) {
    const df t = cf(op, 0);
    const float2 th = f2(t.hi, t.hi), tl = f2(t.lo, t.lo);
    const Cplx u = x;
    if constexpr (MODE == 0) {
      const df t2 = cf(op, 4);
      x = dfc2_sub(u, dfc2_mulv(y, th, tl));
      y = dfc2_add(y, dfc2_mulv(u, f2(t2.hi, t2.hi), f2(t2.lo, t2.lo)));
    } else {
      x = dfc2_sub(dfc2_mulv(u, th, tl), y);
      y = dfc2_add(u, dfc2_mulv(y, th, tl));
    }
  }
  __device__ static Cplx negate(const Cplx& v) {
    return dfc2{mul2(v.hi, f2(-1.f, -1.f)), mul2(v.lo, f2(-1.f, -1.f))};
  }
  __device__ static Cplx scale(const Cplx& v, const FOp& op, int e) {
    const df f = cf(op, e);
    return dfc2_mulv(v, f2(f.hi, f.hi), f2(f.lo, f.lo));
  }
  // (x + r y, y + r x), r = c0
  __device__ static void depol_mix(Cplx& x, Cplx& y, const FOp& op) {
    const df r = cf(op, 0);
    const float2 rh = f2(r.hi, r.hi), rl = f2(r.lo, r.lo);
    const Cplx x0 = x;
    x = dfc2_add(x0, dfc2_mulv(y, rh, rl));
    y = dfc2_add(y, dfc2_mulv(x0, rh, rl));
  }
};

// ------------------------------------------------------------ register ops
template <class A, int R, int K, bool CONJ, bool MASKED, int I>
__device__ __forceinline__ void pair_on_bit(typename A::Cplx (&v)[1 << R], uint32_t rmask,
                                            const FOp& op) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j) {
    if (j & (1 << I)) continue;
    if (MASKED && (uint32_t(j) & rmask) != rmask) continue;
    A::template pair_t<K, CONJ>(v[j], v[j | (1 << I)], op);
  }
}

// Unscaled H / sqrt(X) / sqrt(Y) on register bit I with a real factor c0 on
// the input whose register bit J differs from its bit I: the bit-1 input y
// where bit J is 0, the bit-0 input x where bit J is 1.  With I, J a density
// matrix's row and column bits of one qubit these are exactly the entries
// off the qubit's diagonal: the update applies a deferred off-diagonal
// factor for free (the planner's channel deferral).
template <class A, int R, int K, bool CONJ, int I, int J>
__device__ __forceinline__ void pair_side_on_bit(typename A::Cplx (&v)[1 << R], const FOp& op) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j) {
    if (j & (1 << I)) continue;
    if (j & (1 << J)) A::template pair_xs<K, CONJ>(v[j], v[j | (1 << I)], op);
    else A::template pair_t<K, CONJ>(v[j], v[j | (1 << I)], op);
  }
}

// Phase on the amplitudes with register bit I set: a compile-time set, so no
// lane issues a predicated-off multiply.
template <class A, int R, int I>
__device__ __forceinline__ void phase_on_bit(typename A::Cplx (&v)[1 << R], const FOp& op) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j)
    if (j & (1 << I)) v[j] = A::phase(v[j], op);
}

// Unscaled phase (1 + i t) on the amplitudes with register bit I set.
template <class A, int R, int I>
__device__ __forceinline__ void phaseu_on_bit(typename A::Cplx (&v)[1 << R], const FOp& op) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j)
    if (j & (1 << I)) v[j] = A::phase_u(v[j], op);
}

// Shear along register bit I (MODE as in Arith::shear).
template <class A, int R, int I, int MODE>
__device__ __forceinline__ void shear_on_bit(typename A::Cplx (&v)[1 << R], const FOp& op) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j) {
    if (j & (1 << I)) continue;
    A::template shear<MODE>(v[j], v[j | (1 << I)], op);
  }
}

// i times the amplitudes with register bit I set.
template <class A, int R, int I>
__device__ __forceinline__ void muli_on_bit(typename A::Cplx (&v)[1 << R]) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j)
    if (j & (1 << I)) v[j] = A::mul_i(v[j]);
}

template <class A, int R, int I0, int I1>
__device__ __forceinline__ void depol_on_bits(typename A::Cplx (&v)[1 << R], const FOp& op) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j) {
    if (j & ((1 << I0) | (1 << I1))) continue;
    A::depol_mix(v[j], v[j | (1 << I0) | (1 << I1)], op);
  }
}

// Row / column phase pair on register bits I0 < I1: (1 + i c0) where only
// I0 is set, (1 + i c1) where only I1 is set.
template <class A, int R, int I0, int I1>
__device__ __forceinline__ void offph_on_bits(typename A::Cplx (&v)[1 << R], const FOp& op) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j) {
    const int lo = (j >> I0) & 1, hi = (j >> I1) & 1;
    if (lo && !hi) v[j] = A::template phase_u<0>(v[j], op);
    if (!lo && hi) v[j] = A::template phase_u<1>(v[j], op);
  }
}

// Dephasing-form scale by c0 of the amplitudes whose register bits I0 and I1
// differ (a compile-time half of the register amplitudes).
template <class A, int R, int I0, int I1>
__device__ __forceinline__ void deph_on_bits(typename A::Cplx (&v)[1 << R], const FOp& op) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j)
    if (((j >> I0) ^ (j >> I1)) & 1) v[j] = A::scale(v[j], op, 0);
}


// Operations over a compile-time set M of the register amplitudes (bit j of
// M = amplitude j): the runtime-compiled pass kernels bake each op's set in.
template <class A, int R, uint32_t M>
__device__ __forceinline__ void phase_mask(typename A::Cplx (&v)[1 << R], const FOp& op) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j)
    if ((M >> j) & 1u) v[j] = A::phase(v[j], op);
}
template <class A, int R, uint32_t M>
__device__ __forceinline__ void phaseu_mask(typename A::Cplx (&v)[1 << R], const FOp& op) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j)
    if ((M >> j) & 1u) v[j] = A::phase_u(v[j], op);
}
template <class A, int R, uint32_t M>
__device__ __forceinline__ void muli_mask(typename A::Cplx (&v)[1 << R]) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j)
    if ((M >> j) & 1u) v[j] = A::mul_i(v[j]);
}
template <class A, int R, uint32_t M>
__device__ __forceinline__ void negate_mask(typename A::Cplx (&v)[1 << R]) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j)
    if ((M >> j) & 1u) v[j] = A::negate(v[j]);
}

// Dephasing-form scale by c0 where two index bits differ; each bit comes
// from the register index j (BS_REG), the thread's local index tl
// (BS_LOCAL) or the tile's global base (BS_GLOBAL), at position AP / BP.
template <int S, int P>
__device__ __forceinline__ int src_bit(int j, uint32_t tl, uint64_t base) {
  if constexpr (S == BS_REG) return (j >> P) & 1;
  else if constexpr (S == BS_LOCAL) return int((tl >> P) & 1u);
  else return int((base >> P) & 1u);
}
template <class A, int R, int AS, int AP, int BS, int BP>
__device__ __forceinline__ void deph_src(typename A::Cplx (&v)[1 << R], uint32_t tl, uint64_t base,
                                         const FOp& op) {
#pragma unroll
  for (int j = 0; j < (1 << R); ++j)
    if (src_bit<AS, AP>(j, tl, base) != src_bit<BS, BP>(j, tl, base)) v[j] = A::scale(v[j], op, 0);
}

}  // namespace qs
