// Arithmetic of one 2x2 update on an amplitude pair (Eq. 1), shared by the
// one-pass-per-gate kernels, the fused tile kernel and the runtime-compiled
// pass kernels (so it compiles under NVRTC as well as nvcc).
#pragma once
#include "common.cuh"

namespace qs {

// ---------------------------------------------------------------- pair ops
// Gate classes of the paper's benchmark set (Sec. II.C) with their own
// arithmetic, plus the general 2x2 matrix (Eq. 1).
// The U forms are H, sqrt(X), sqrt(Y) without their scalar factors (1/sqrt 2,
// (1+i)/2, and (1-i)/2 for conjugated column updates), which the register
// then carries (Reg::pend_scale): [[1, 1], [1, -1]], [[1, -i], [-i, 1]]
// (conj: [[1, i], [i, 1]]), [[1, -1], [1, 1]].
enum PairKind { PK_GEN = 0, PK_H = 1, PK_SX = 2, PK_SY = 3, PK_X = 4, PK_HU = 5, PK_SXU = 6, PK_SYU = 7,
                PK_PSP = 8, PK_PSP2 = 9 };

// (x, y) <- G (x, y); CONJ applies conj(G) instead (Eq. 2 column update).
template <typename R, int K, bool CONJ>
__device__ __forceinline__ void pair_apply(cvec<R>& x, cvec<R>& y, const Mat2<R>& g) {
  const R xr = x.x, xi = x.y, yr = y.x, yi = y.y;
  if constexpr (K == PK_GEN) {
    const R s = CONJ ? R(-1) : R(1);
    const R i0 = s * g.im[0], i1 = s * g.im[1], i2 = s * g.im[2], i3 = s * g.im[3];
    // explicit FMA chains (one product rounded, three fused): the same
    // rounding in every kernel that includes this, whatever the compiler's
    // contraction choices
    x.x = fma(g.re[0], xr, fma(-i0, xi, fma(g.re[1], yr, -(i1 * yi))));
    x.y = fma(g.re[0], xi, fma(i0, xr, fma(g.re[1], yi, i1 * yr)));
    y.x = fma(g.re[2], xr, fma(-i2, xi, fma(g.re[3], yr, -(i3 * yi))));
    y.y = fma(g.re[2], xi, fma(i2, xr, fma(g.re[3], yi, i3 * yr)));
  } else if constexpr (K == PK_H) {
    // H = [[1, 1], [1, -1]] / sqrt(2); real, so conj(H) = H.  g.re[0] = 1/sqrt(2).
    const R s = g.re[0];
    x.x = (xr + yr) * s; x.y = (xi + yi) * s;
    y.x = (xr - yr) * s; y.y = (xi - yi) * s;
  } else if constexpr (K == PK_SX) {
    // sqrt(X) = [[1+i, 1-i], [1-i, 1+i]] / 2:  with u = x + y, v = x - y,
    // x' = (u + i v) / 2, y' = (u - i v) / 2  (conj swaps the two signs).
    const R ur = (xr + yr) * R(0.5), ui = (xi + yi) * R(0.5);
    const R vr = (xr - yr) * R(0.5), vi = (xi - yi) * R(0.5);
    if constexpr (!CONJ) {
      x.x = ur - vi; x.y = ui + vr; y.x = ur + vi; y.y = ui - vr;
    } else {
      x.x = ur + vi; x.y = ui - vr; y.x = ur - vi; y.y = ui + vr;
    }
  } else if constexpr (K == PK_SY) {
    // sqrt(Y) = w [[1, -1], [1, 1]], w = (1+i)/2:  x' = w (x - y), y' = w (x + y);
    // w z = ((zr - zi) + i (zr + zi)) / 2,  conj(w) z = ((zr + zi) + i (zi - zr)) / 2.
    const R dr = xr - yr, di = xi - yi, sr = xr + yr, si = xi + yi;
    if constexpr (!CONJ) {
      x.x = (dr - di) * R(0.5); x.y = (dr + di) * R(0.5);
      y.x = (sr - si) * R(0.5); y.y = (sr + si) * R(0.5);
    } else {
      x.x = (dr + di) * R(0.5); x.y = (di - dr) * R(0.5);
      y.x = (sr + si) * R(0.5); y.y = (si - sr) * R(0.5);
    }
  } else if constexpr (K == PK_X) {
    x.x = yr; x.y = yi; y.x = xr; y.y = xi;
  } else if constexpr (K == PK_HU) {  // unscaled, bit-1 input times c = g.re[0] (FMA: free)
    const R c = g.re[0];
    x.x = fma(c, yr, xr); x.y = fma(c, yi, xi); y.x = fma(-c, yr, xr); y.y = fma(-c, yi, xi);
  } else if constexpr (K == PK_SXU) {
    const R c = g.re[0];
    if constexpr (!CONJ) {
      x.x = fma(c, yi, xr); x.y = fma(-c, yr, xi); y.x = fma(c, yr, xi); y.y = fma(c, yi, -xr);
    } else {
      x.x = fma(-c, yi, xr); x.y = fma(c, yr, xi); y.x = fma(c, yr, -xi); y.y = fma(c, yi, xr);
    }
  } else if constexpr (K == PK_SYU) {
    const R c = g.re[0];
    x.x = fma(-c, yr, xr); x.y = fma(-c, yi, xi); y.x = fma(c, yr, xr); y.y = fma(c, yi, xi);
  } else if constexpr (K == PK_PSP || K == PK_PSP2) {
    // a general update as phase-shear with deferred factors (launch.cu):
    // y~ = (1 + i t2) y (PSP) or (t2 + i) y (PSP2), then (x - a1 y~, y~ + a2 x);
    // g.re = {t2, a1, a2}
    const R t2 = g.re[0], a1 = g.re[1], a2 = g.re[2];
    const R zr = K == PK_PSP ? fma(-t2, yi, yr) : fma(t2, yr, -yi);
    const R zi = K == PK_PSP ? fma(t2, yr, yi) : fma(t2, yi, yr);
    x.x = fma(-a1, zr, xr); x.y = fma(-a1, zi, xi);
    y.x = fma(a2, xr, zr); y.y = fma(a2, xi, zi);
  }
}

}  // namespace qs
