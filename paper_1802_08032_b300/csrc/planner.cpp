// Fusion planner: gate list -> fused passes of encoded operations.
//
// Planner.  Gates are first expanded into vector operations on the stored
// 2^nq vector (a density-matrix gate G on qubit t becomes G on bit t and
// conj(G) on bit t+N, Eq. 2).  Each operation has X bits (where it mixes
// amplitudes: the target of a pair update, both bits of a depolarising
// quad) and Z bits (where it only reads the index: controls, the bits of
// diagonal operations).  A pass takes operations in order while their X
// bits fit in the k tile qubits; an operation that does not fit is
// deferred, and a later operation may move ahead of deferred ones only if
// it commutes with all of them (no X bit of either touches a bit of the
// other).  Several candidate tiles compete for each pass (see plan()).
// Passes repeat until the queue is empty.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

#include "plan.h"
#include "runtime.h"

namespace qs {

namespace {

struct VOp {
  FKind kind;
  bool conj = false;
  bool spread = false;   // H / sqrt(X) / sqrt(Y) on a bit whose bit-1 amplitudes are all 0
  int b0 = -1, b1 = -1;  // pair target (b0); DEPOL row/column; DEPH the two compared bits
  int side = -1;         // H / sqrt(X) / sqrt(Y): c0 scales the input whose bit `side` differs from its bit b0
  uint64_t cond = 0;     // bits that must all be 1 (controls; PHASE/SIGN diagonal support)
  double c[8] = {};

  uint64_t xmask() const {
    // (a side factor's bit joins the tile and the register bits with b0)
    if (side >= 0) return (uint64_t(1) << b0) | (uint64_t(1) << side);
    if (kind <= FK_X || kind == FK_SHEAR) return uint64_t(1) << b0;
    // (a row / column phase pair is diagonal, but it must run on register
    // bits: counting its bits as moved keeps them in the tile)
    if (kind == FK_DEPOL || kind == FK_OFFPH) return (uint64_t(1) << b0) | (uint64_t(1) << b1);
    return 0;
  }
  uint64_t zmask() const {
    uint64_t z = cond;
    if (kind == FK_DEPH) z |= (uint64_t(1) << b0) | (uint64_t(1) << b1);
    return z;
  }
};

VOp pair_op(OpK k, int bit, uint64_t cond, const double* m, bool conj) {
  VOp v;
  v.kind = FKind(int(k));  // GEN..X share the numbering
  v.b0 = bit;
  v.cond = cond;
  v.conj = conj;
  if (k == OpK::GEN) std::memcpy(v.c, m, sizeof(v.c));
  if (k == OpK::H || k == OpK::SX || k == OpK::SY) v.c[0] = 1.0;  // factor on the bit-1 input
  if (cond != 0 && (k == OpK::H || k == OpK::SX || k == OpK::SY)) {
    // the engine applies these unscaled (a global factor), which a control
    // would break: use the explicit matrix instead
    const double h = std::sqrt(0.5);
    const double H[8] = {h, 0, h, 0, h, 0, -h, 0};
    const double SX[8] = {0.5, 0.5, 0.5, -0.5, 0.5, -0.5, 0.5, 0.5};
    const double SY[8] = {0.5, 0.5, -0.5, -0.5, 0.5, 0.5, 0.5, 0.5};
    const double* src = k == OpK::H ? H : (k == OpK::SX ? SX : SY);
    for (int e = 0; e < 8; ++e) v.c[e] = src[e];
    v.kind = FK_GEN;
  }
  return v;
}

void expand(const Reg& r, const GateOp& op, std::vector<VOp>& out) {
  const int N = r.n;
  switch (op.k) {
    case OpK::GEN: case OpK::H: case OpK::SX: case OpK::SY: case OpK::X:
      out.push_back(pair_op(op.k, op.t, op.cmask, op.m, false));
      if (r.density) out.push_back(pair_op(op.k, op.t + N, op.cmask << N, op.m, true));
      return;
    case OpK::PHASE: {
      VOp v;
      v.kind = FK_PHASE;
      v.cond = op.cmask | (uint64_t(1) << op.t);
      v.c[0] = op.m[0];
      v.c[1] = op.m[1];
      out.push_back(v);
      if (r.density) {  // column factor e^{-i phi}
        v.cond <<= N;
        v.c[1] = -op.m[1];
        out.push_back(v);
      }
      return;
    }
    case OpK::SIGN: {
      VOp v;
      v.kind = FK_SIGN;
      v.cond = op.cmask;
      out.push_back(v);
      if (r.density) {
        v.cond <<= N;
        out.push_back(v);
      }
      return;
    }
    case OpK::DEPHASE: {
      VOp v;
      v.kind = FK_DEPH;
      v.b0 = op.t;
      v.b1 = op.t + N;
      v.c[0] = 1.0 - 2.0 * op.m[0];
      out.push_back(v);
      return;
    }
    case OpK::MULTI:
      fail(QS_E_ARG, "multi-target gates are not planned into fused passes");
    case OpK::DEPOL: {
      const double p = op.m[0];
      VOp v;
      v.kind = FK_DEPOL;
      v.b0 = op.t;
      v.b1 = op.t + N;
      v.c[0] = 1.0 - 2.0 * p / 3.0;
      v.c[1] = 2.0 * p / 3.0;
      v.c[2] = 1.0 - 4.0 * p / 3.0;
      out.push_back(v);
      return;
    }
  }
}

// Appends FK_SCALE operations carrying the factors that the engine's
// unscaled H / sqrt(X) / sqrt(Y) leave out (1/sqrt 2, (1+i)/2, and (1-i)/2
// for conjugated column updates).  Every operation is linear, so the factor
// is carried across the passes of a plan and applied once, in its last
// pass, or earlier whenever the pending magnitude growth 2^(e/2) reaches the
// arithmetic's limit (2^40 for float exponents, 2^500 for FP64).
// The product of e dropped factors, p of them (1+i)/2 and q of them (1-i)/2,
// is 2^(-e/2) e^{i pi (p-q)/4}; it is formed directly (at most one rounding,
// in 1/sqrt 2) rather than by e successive multiplications.
std::complex<double> dropped_factor(int e, int p, int q) {
  const int k = ((p - q) % 8 + 8) % 8;
  const double s = std::sqrt(0.5);
  const double mag = std::ldexp(1.0, -(e / 2));
  // e^{i pi k / 4} with exact components for even k
  static const int re_sign[8] = {1, 1, 0, -1, -1, -1, 0, 1};
  static const int im_sign[8] = {0, 1, 1, 1, 0, -1, -1, -1};
  const bool odd_e = e & 1, odd_k = k & 1;
  // |component| of the unit phase is 1 (even k, nonzero) or 1/sqrt 2 (odd k)
  double c = mag;
  if (odd_e && odd_k) c *= 0.5;
  else if (odd_e || odd_k) c *= s;
  return {re_sign[k] * c, im_sign[k] * c};
}

struct ScaleState {
  int e = 0, p = 0, q = 0;
  std::complex<double> g{1.0, 0.0};  // factors left out by shears (see decompose_general)
  int shears = 0;                    // their growth, at most sqrt 2 each
  int limit = 80;
};

void add_scales(std::vector<VOp>& ops, ScaleState& st, bool last) {
  std::vector<VOp> out;
  out.reserve(ops.size() + 2);
  int &e = st.e, &p = st.p, &q = st.q;
  auto flush_scale = [&] {
    if (e == 0 && st.g == std::complex<double>(1.0, 0.0)) {
      st.shears = 0;
      return;
    }
    const std::complex<double> f = dropped_factor(e, p, q) * st.g;
    st.g = 1.0;
    st.shears = 0;
    VOp s;
    s.kind = FK_SCALE;
    s.c[0] = f.real();
    s.c[1] = f.imag();
    out.push_back(s);
    e = p = q = 0;
  };
  for (const VOp& v : ops) {
    out.push_back(v);
    if (v.kind == FK_H) {
      ++e;
    } else if (v.kind == FK_SX || v.kind == FK_SY) {
      ++e;
      if (v.conj) ++q;
      else ++p;
    } else if (v.kind == FK_SHEAR) {
      ++st.shears;
      st.g *= std::complex<double>(v.c[2], v.c[3]);
    }
    if (e + st.shears >= st.limit) flush_scale();
  }
  if (last) flush_scale();
  ops.swap(out);
}

struct Pass {
  std::vector<int> q;  // tile qubits, ascending
  std::vector<VOp> ops;
};

// Bits known to hold only zeros (every amplitude with the bit set is 0, see
// Reg::zero_bits) simplify what follows: a phase, sign flip or
// multiplication by i conditioned on such a bit touches only zeros and is
// dropped, as is a dephasing whose two bits are both such bits and a pair
// update with such a bit among its controls; H, sqrt(X) and sqrt(Y) on such
// a bit map (x, 0) to (x, x), (x, -i x) or (x, i x) (unscaled): the op is
// marked as a copy (made when its stage loads the amplitudes) followed, for
// sqrt(X), by a multiplication by i and (for -i) a sign flip on the bit.
// Every operation that mixes amplitudes along a bit clears it.
void apply_zero_bits(std::vector<VOp>& ops, uint64_t& zero) {
  std::vector<VOp> out;
  out.reserve(ops.size());
  for (VOp v : ops) {
    const uint64_t x = v.xmask();
    if (v.kind == FK_PHASE || v.kind == FK_SIGN || v.kind == FK_MULI) {
      if ((v.cond & zero) == 0) out.push_back(v);
      continue;
    }
    if (v.kind == FK_DEPH) {
      const uint64_t both = (uint64_t(1) << v.b0) | (uint64_t(1) << v.b1);
      if ((zero & both) != both) out.push_back(v);
      continue;
    }
    if (v.kind <= FK_X) {
      if (v.cond & zero) continue;
      if ((zero & x) && v.cond == 0 && (v.kind == FK_H || v.kind == FK_SX || v.kind == FK_SY)) {
        v.spread = true;
        zero &= ~x;
        out.push_back(v);
        if (v.kind == FK_SX) {
          VOp m;
          m.kind = FK_MULI;
          m.cond = x;
          out.push_back(m);
          if (!v.conj) {
            m.kind = FK_SIGN;
            out.push_back(m);
          }
        }
        continue;
      }
    }
    zero &= ~x;
    out.push_back(v);
  }
  ops.swap(out);
}

// Consecutive phases on one bit merge into one operation (T^2 = S is a
// multiplication by i, T^4 = Z a sign flip: neither needs arithmetic).  A
// phase on a single bit commutes with every operation except those that
// mix amplitudes along that bit (a pair update on it, a depolarising quad
// on it), so it is carried forward to the next such operation, or to the
// end, and emitted there.  T factors (1 + i)/sqrt 2 and their conjugates
// (density-matrix column updates) are counted exactly as multiples k of
// pi/4: k = 4 is a sign flip, k = 2 a multiplication by i, k = 6 both, odd k
// one phase with components +-1/sqrt 2; any other phase joins one general
// factor, multiplied out once.
void merge_phases(std::vector<VOp>& ops, int nq) {
  struct Pending {
    int k = 0;
    std::complex<double> g{1.0, 0.0};
    bool general = false, any = false;
  };
  const double s = std::sqrt(0.5);
  static const double ur[8] = {1, s, 0, -s, -1, -s, 0, s}, ui[8] = {0, s, 1, s, 0, -s, -1, -s};
  std::vector<Pending> pend(static_cast<size_t>(nq));
  std::vector<VOp> out;
  out.reserve(ops.size());
  auto emit = [&](int b) {
    Pending& p = pend[size_t(b)];
    if (!p.any) return;
    const uint64_t bit = uint64_t(1) << b;
    const int k = ((p.k % 8) + 8) % 8;
    VOp v;
    v.cond = bit;
    if (p.general || (k & 1)) {
      const std::complex<double> f = p.g * std::complex<double>(ur[k], ui[k]);
      v.kind = FK_PHASE;
      v.c[0] = p.general ? f.real() : ur[k];
      v.c[1] = p.general ? f.imag() : ui[k];
      out.push_back(v);
    } else if (k == 2 || k == 6) {
      v.kind = FK_MULI;
      out.push_back(v);
      if (k == 6) {
        v.kind = FK_SIGN;
        out.push_back(v);
      }
    } else if (k == 4) {
      v.kind = FK_SIGN;
      out.push_back(v);
    }
    p = Pending{};
  };
  for (const VOp& v : ops) {
    if (v.kind == FK_PHASE && __builtin_popcountll(v.cond) == 1) {
      Pending& p = pend[size_t(__builtin_ctzll(v.cond))];
      p.any = true;
      if (v.c[0] == s && v.c[1] == s) {
        p.k += 1;
      } else if (v.c[0] == s && v.c[1] == -s) {
        p.k -= 1;
      } else {
        p.g *= std::complex<double>(v.c[0], v.c[1]);
        p.general = true;
      }
      continue;
    }
    const uint64_t x = v.xmask();
    for (int b = 0; b < nq; ++b)
      if ((x >> b) & 1) emit(b);
    out.push_back(v);
  }
  for (int b = 0; b < nq; ++b) emit(b);
  ops.swap(out);
}

// The 2x2 matrix an op applies along bit b (row-major), when it is a
// single-bit unitary acting on b alone: an uncontrolled pair update on b
// (true matrices, with the scale factors the engine's H / sqrt(X) / sqrt(Y)
// leave out; conjugated for density-matrix column updates) or a phase,
// multiplication by i or sign flip conditioned on b alone.
bool single_bit_matrix(const VOp& v, int b, std::complex<double> m[4]) {
  using C = std::complex<double>;
  const uint64_t bit = uint64_t(1) << b;
  if (v.kind <= FK_SY && v.cond == 0 && v.b0 == b && !v.spread) {
    const double s = std::sqrt(0.5);
    if (v.kind == FK_GEN) {
      for (int e = 0; e < 4; ++e) m[e] = C(v.c[2 * e], v.c[2 * e + 1]);
    } else if (v.kind == FK_H) {
      m[0] = s; m[1] = s; m[2] = s; m[3] = -s;
    } else if (v.kind == FK_SX) {
      m[0] = C(0.5, 0.5); m[1] = C(0.5, -0.5); m[2] = C(0.5, -0.5); m[3] = C(0.5, 0.5);
    } else {  // sqrt(Y)
      m[0] = C(0.5, 0.5); m[1] = C(-0.5, -0.5); m[2] = C(0.5, 0.5); m[3] = C(0.5, 0.5);
    }
    if (v.conj)
      for (int e = 0; e < 4; ++e) m[e] = std::conj(m[e]);
    return true;
  }
  if (v.cond == bit && (v.kind == FK_PHASE || v.kind == FK_MULI || v.kind == FK_SIGN)) {
    m[0] = 1;
    m[1] = 0;
    m[2] = 0;
    m[3] = v.kind == FK_PHASE ? C(v.c[0], v.c[1]) : (v.kind == FK_MULI ? C(0, 1) : C(-1, 0));
    return true;
  }
  return false;
}

// An uncontrolled general 2x2 update absorbs the single-bit unitaries just
// before it on its bit (every op in between leaves the bit alone, so they
// commute): one general update costs the same as before, the absorbed ops
// cost nothing.
void absorb_into_general(std::vector<VOp>& ops) {
  using C = std::complex<double>;
  std::vector<bool> dead(ops.size(), false);
  for (size_t i = 0; i < ops.size(); ++i) {
    VOp& g = ops[i];
    if (g.kind != FK_GEN || g.cond != 0) continue;
    const int b = g.b0;
    const uint64_t bit = uint64_t(1) << b;
    C G[4];
    single_bit_matrix(g, b, G);
    bool changed = false;
    for (size_t j = i; j-- > 0;) {
      if (dead[j] || ((ops[j].xmask() | ops[j].zmask()) & bit) == 0) continue;
      C M[4];
      if (!single_bit_matrix(ops[j], b, M)) break;
      const C P[4] = {G[0] * M[0] + G[1] * M[2], G[0] * M[1] + G[1] * M[3],
                      G[2] * M[0] + G[3] * M[2], G[2] * M[1] + G[3] * M[3]};
      for (int e = 0; e < 4; ++e) G[e] = P[e];
      dead[j] = true;
      changed = true;
    }
    if (changed) {
      for (int e = 0; e < 4; ++e) {
        g.c[2 * e] = G[e].real();
        g.c[2 * e + 1] = G[e].imag();
      }
      g.conj = false;
    }
  }
  size_t w = 0;
  for (size_t i = 0; i < ops.size(); ++i)
    if (!dead[i]) ops[w++] = ops[i];
  ops.resize(w);
}

// An uncontrolled general 2x2 update U = [[a, b], [c, d]] factors exactly as
// g diag(1, p1) R diag(1, p2), with unit phases g = a/|a|,
// p1 = (c/|c|) conj(g), p2 = -(b/|b|) conj(g) and the real rotation
// R = [[|a|, -|b|], [|b|, |a|]] = m [[1, -t], [t, 1]] (m = |a| >= |b|,
// t = |b|/|a|) or m [[t, -1], [1, t]] (m = |b|, t = |a|/|b|).  The rotation
// runs as a shear with one FMA per output component and g m joins the
// factors applied once per plan; the two phases cost what half a general
// update does and may merge with neighbouring phases.  Together: 12 FP64
// operations per pair instead of 16.  Matrices whose factors do not
// reproduce them to 1e-14 (not unitary to that precision, or |a| or |b| 0)
// stay general.
// max_t: the largest t the first form may take (its deferred factor |a|
// then is at least 1/sqrt(1 + max_t^2)).
void decompose_general(std::vector<VOp>& ops, double max_t) {
  using C = std::complex<double>;
  std::vector<VOp> out;
  out.reserve(ops.size() + ops.size() / 2);
  for (const VOp& v : ops) {
    if (v.kind != FK_GEN || v.cond != 0) {
      out.push_back(v);
      continue;
    }
    C U[4];
    single_bit_matrix(v, v.b0, U);
    const double na = std::abs(U[0]), nb = std::abs(U[1]), nc = std::abs(U[2]);
    if (!(na > 1e-150 && nb > 1e-150 && nc > 1e-150)) {
      out.push_back(v);
      continue;
    }
    const C g = U[0] / na, p1 = (U[2] / nc) * std::conj(g), p2 = -(U[1] / nb) * std::conj(g);
    // reproduce U from the factors (R uses |b| for both off-diagonal magnitudes)
    const C r01 = -g * nb * p2, r10 = g * p1 * nb, r11 = g * p1 * na * p2;
    if (std::abs(r01 - U[1]) > 1e-14 || std::abs(r10 - U[2]) > 1e-14 || std::abs(r11 - U[3]) > 1e-14) {
      out.push_back(v);
      continue;
    }
    const uint64_t bit = uint64_t(1) << v.b0;
    auto phase = [&](C z) {
      if (z == C(1.0, 0.0)) return;
      VOp ph;
      ph.kind = FK_PHASE;
      ph.cond = bit;
      ph.c[0] = z.real();
      ph.c[1] = z.imag();
      out.push_back(ph);
    };
    phase(p2);
    VOp sh;
    sh.kind = FK_SHEAR;
    sh.b0 = v.b0;
    const bool by_a = na * max_t >= nb;
    sh.c[0] = by_a ? nb / na : na / nb;  // t <= max_t (first form) or < 1
    sh.c[1] = by_a ? 0.0 : 1.0;          // form
    sh.c[4] = sh.c[0];
    const C f = g * (by_a ? na : nb);
    sh.c[2] = f.real();
    sh.c[3] = f.imag();
    out.push_back(sh);
    phase(p1);
  }
  ops.swap(out);
}

// A phase e^{i psi} = cos psi (1 + i tan psi) on a single bit: the bracket
// costs one FMA per output component (2 per touched amplitude, against 4
// for the complex product), and the real factor c = cos psi, which
// multiplies every amplitude with the bit set, commutes with everything up
// to the next operation that mixes amplitudes along the bit.  When that
// operation is an uncontrolled H / sqrt(X) / sqrt(Y), it takes the factor on
// its bit-1 input at no cost (its additions become FMAs).  A first-form
// shear (x - t y, y + t' x) on the bit lets the factor through, also at no
// cost: with y = c y~ it computes x - (t c) y~ and y~ + (t'/c) x, the factor
// staying on the bit-1 half.  Only for plain FP32 / FP64 arithmetic (a
// double-float scaled add is not free), and only for |cos psi| >= 1/4,
// which bounds the growth.
void unscale_phases(std::vector<VOp>& ops) {
  std::vector<size_t> through;
  for (size_t i = 0; i < ops.size(); ++i) {
    VOp& ph = ops[i];
    if (ph.kind != FK_PHASE || __builtin_popcountll(ph.cond) != 1 || !(std::fabs(ph.c[0]) >= 0.25)) continue;
    const uint64_t bit = ph.cond;
    through.clear();
    for (size_t j = i + 1; j < ops.size(); ++j) {
      if ((ops[j].xmask() & bit) == 0) continue;
      VOp& p = ops[j];
      if (p.kind == FK_SHEAR && p.c[1] == 0.0) {
        through.push_back(j);
        continue;
      }
      if ((p.kind == FK_H || p.kind == FK_SX || p.kind == FK_SY) && p.cond == 0 && !p.spread) {
        const double c = ph.c[0];
        for (size_t t : through) {
          ops[t].c[0] *= c;
          ops[t].c[4] /= c;
        }
        p.c[0] *= c;
        ph.kind = FK_PHASEU;
        ph.c[0] = ph.c[1] / c;
        ph.c[1] = 0.0;
      }
      break;
    }
  }
}

// Channels on a density matrix (Eq. 2 vectorisation: row bit t, column bit
// t + N).  A dephasing scales the entries whose row and column bits differ
// (the off-diagonal ones in t) by 1 - 2p; a depolarising channel scales them
// by 1 - 4p/3 and mixes the diagonal pair (x, y) into ((1 - m) x + m y,
// m x + (1 - m) y), m = 2p/3.  Written as
//   (1 - m) * [ off -> (s / (1 - m)) off,  (x, y) -> (x + r y, y + r x) ],
// r = m / (1 - m), the common factor 1 - m joins the plan's final scale and
// the off-diagonal factor is kept per qubit, F[t]: an entrywise real scale
// commutes with every operation that does not mix amplitudes along bit t or
// t + N (diagonal ops; pair updates, depolarising mixes and dephasings on
// other qubits move or mix entries with equal bits t and t + N; a
// depolarising mix on t itself moves only diagonal entries).  So consecutive
// channels on t multiply into F[t], which one dephasing-form op applies just
// before the next pair update on t or t + N, or at the end of the plan.  The
// depolarising op left in the list is the diagonal mix alone (4 FMAs a quad
// instead of 10 operations).  Returns the common factor; a FK_SCALE carries
// it earlier if it falls below 2^-30.
// A gate's phase e^{i phi} on row bit t and its conjugate on column bit t + N
// (Eq. 2) cancel on the diagonal entries and give e^{+-i phi} on the two
// off-diagonal halves: when nothing between them moves amplitudes along t or
// t + N, the two phases become one op, (1 +- i tan phi) on the off-diagonal
// entries only, and cos phi joins F[t].
// With FP64 arithmetic an uncontrolled H / sqrt(X) / sqrt(Y) on t or t + N
// (bit-1 factor 1) takes F[t] itself: its inputs off the qubit's diagonal
// are the bit-1 one where the partner bit is 0 and the bit-0 one where it is
// 1, and the kernel scales whichever it is inside the update's FMAs.
double defer_offdiag(std::vector<VOp>& ops, int N, bool side_factors) {
  std::vector<double> F(size_t(N), 1.0);
  double G = 1.0;
  std::vector<VOp> out;
  out.reserve(ops.size() + size_t(N));
  auto settle = [&](int t) {
    if (F[size_t(t)] == 1.0) return;
    VOp d;
    d.kind = FK_DEPH;
    d.b0 = t;
    d.b1 = t + N;
    d.c[0] = F[size_t(t)];
    out.push_back(d);
    F[size_t(t)] = 1.0;
  };
  std::vector<bool> used(ops.size(), false);
  for (size_t i = 0; i < ops.size(); ++i) {
    const VOp& v = ops[i];
    if (used[i]) continue;
    if (v.kind == FK_DEPH) {
      F[size_t(v.b0)] *= v.c[0];
      continue;
    }
    if (v.kind == FK_PHASE && __builtin_popcountll(v.cond) == 1 && __builtin_ctzll(v.cond) < N &&
        std::abs(v.c[0]) >= 0.5) {
      const int t = __builtin_ctzll(v.cond);
      const uint64_t col = uint64_t(1) << (t + N), both = v.cond | col;
      // (the two are normally adjacent; the search is capped so that a long
      // run of unrelated ops keeps planning linear)
      size_t j = i + 1;
      const size_t jmax = std::min(ops.size(), i + 64);
      for (; j < jmax; ++j) {
        const VOp& w = ops[j];
        if (!used[j] && w.kind == FK_PHASE && w.cond == col) break;
        if (w.xmask() & both) {
          j = jmax;
          break;
        }
      }
      if (j == jmax) j = ops.size();
      if (j < ops.size() && ops[j].c[0] == v.c[0] && ops[j].c[1] == -v.c[1]) {
        used[j] = true;
        F[size_t(t)] *= v.c[0];
        VOp o;
        o.kind = FK_OFFPH;
        o.b0 = t;
        o.b1 = t + N;
        o.c[0] = v.c[1] / v.c[0];  // where row bit = 1, column bit = 0
        o.c[1] = -o.c[0];
        out.push_back(o);
        continue;
      }
    }
    if (v.kind == FK_DEPOL) {
      const double keep = v.c[0], move = v.c[1], off = v.c[2];
      F[size_t(v.b0)] *= off / keep;
      G *= keep;
      VOp d = v;
      d.c[0] = move / keep;
      d.c[1] = d.c[2] = 0.0;
      out.push_back(d);
      if (G < 0x1p-30) {
        VOp sc;
        sc.kind = FK_SCALE;
        sc.c[0] = G;
        out.push_back(sc);
        G = 1.0;
      }
      continue;
    }
    const uint64_t x = v.xmask();
    if (side_factors && (v.kind == FK_H || v.kind == FK_SX || v.kind == FK_SY) && v.cond == 0 && !v.spread &&
        v.c[0] == 1.0) {
      const int t = v.b0 < N ? v.b0 : v.b0 - N;
      if (F[size_t(t)] != 1.0) {
        VOp w = v;
        w.side = v.b0 < N ? t + N : t;
        w.c[0] = F[size_t(t)];
        F[size_t(t)] = 1.0;
        out.push_back(w);
        continue;
      }
    }
    for (int t = 0; t < N; ++t)
      if (((x >> t) | (x >> (t + N))) & 1) settle(t);
    out.push_back(v);
  }
  for (int t = 0; t < N; ++t) settle(t);
  ops.swap(out);
  return G;
}

int popc(uint64_t x) { return __builtin_popcountll(x); }

std::vector<Pass> plan(const std::vector<VOp>& ops, int nq, int k, int L, int64_t max_ops,
                       int scale_limit, std::complex<double> scale_in, int dm_n) {
  std::vector<Pass> passes;
  std::vector<VOp> rem = ops;
  ScaleState scale;
  scale.limit = scale_limit;
  scale.g = scale_in;
  const uint64_t low = (uint64_t(1) << L) - 1;
  const uint64_t all = nq >= 64 ? ~uint64_t(0) : (uint64_t(1) << nq) - 1;
  // One candidate pass: the tile starts as T0 and, with grow, takes the X
  // bits of each op that still fits in k qubits; an op is taken if its X
  // bits are in the tile and it commutes with every op deferred so far.
  auto simulate = [&](uint64_t T0, bool grow, Pass& p, std::vector<VOp>& deferred, uint64_t& tile) {
    tile = T0;
    uint64_t bx = 0, ball = 0;
    p.ops.clear();
    deferred.clear();
    for (const VOp& v : rem) {
      const uint64_t x = v.xmask(), z = v.zmask();
      // A mid-plan scale (a density matrix's deferred channel factor)
      // balances the growth of the operations before it; moved ahead of a
      // deferred one it would shrink the amplitudes early, and with float
      // exponents (double-float) values below 2^-74 lose their low parts
      // when a pass boundary stores them.  So it stays behind every deferred
      // op, and no later op that mixes amplitudes passes it.
      if (v.kind == FK_SCALE && !deferred.empty()) {
        deferred.push_back(v);
        ball = all;
        continue;
      }
      const bool commutes = (x & ball) == 0 && ((x | z) & bx) == 0;
      const bool fits = grow ? popc(tile | x) <= k : (x & ~tile) == 0;
      const bool room = int64_t(p.ops.size()) < max_ops;
      if (commutes && fits && room) {
        tile |= x;
        p.ops.push_back(v);
      } else {
        deferred.push_back(v);
        bx |= x;
        ball |= x | z;
      }
    }
  };
  auto moving = [](const Pass& p) {
    int c = 0;
    for (const VOp& v : p.ops) c += v.xmask() != 0;
    return c;
  };
  while (!rem.empty()) {
    Pass p, cp;
    std::vector<VOp> deferred, cdef;
    uint64_t tile = 0, ctile = 0;
    // Candidate tiles: the one grown from the ops in order, and the low L
    // qubits plus a window of adjacent qubits (a density matrix: a block of
    // rows with its column partners, bit t + N, topped up from the ops).
    // On layered circuits a block of neighbouring qubits can advance several
    // layers in one pass, bounded by its neighbours, where the first ops'
    // qubits are scattered across a layer.  The candidate taking the most
    // ops that move amplitudes wins (ties: the grown tile, then the lower
    // window).  30-qubit workload: 28 -> 19 passes (complex64, k = 12),
    // 26 -> 19 (complex128); 14-qubit noisy density matrix 18 -> 15.
    simulate(low, true, p, deferred, tile);
    int best = moving(p);
    std::vector<uint64_t> cands;
    const int w = k - L;
    if (dm_n == 0) {
      for (int b = L; w > 0 && b + w <= nq; ++b) cands.push_back(low | (((uint64_t(1) << w) - 1) << b));
    } else {
      // a block of rows with its column partners (bit t + N)
      for (int h = 1; 2 * h <= k; ++h)
        for (int b = 0; b + h <= dm_n; ++b) {
          const uint64_t rows = ((uint64_t(1) << h) - 1) << b;
          const uint64_t T = low | rows | (rows << dm_n);
          if (popc(T) <= k) cands.push_back(T);
        }
    }
    for (uint64_t T : cands) {
      simulate(T, popc(T) < k, cp, cdef, ctile);
      if (cp.ops.empty()) continue;  // (each pass must take an op)
      const int m = moving(cp);
      if (m > best) {
        best = m;
        std::swap(p, cp);
        deferred.swap(cdef);
        tile = ctile;
      }
    }
    // pad the tile to exactly k qubits with the lowest unused ones
    for (int b = 0; b < nq && popc(tile) < k; ++b) tile |= uint64_t(1) << b;
    for (int b = 0; b < nq; ++b)
      if ((tile >> b) & 1) p.q.push_back(b);
    add_scales(p.ops, scale, deferred.empty());
    passes.push_back(std::move(p));
    rem.swap(deferred);
  }
  return passes;
}

void set_coeffs(FOp& f, const double* c, Arith a) {
  for (int e = 0; e < 8; ++e) {
    if (a == Arith::F64) {
      f.c.d[e] = c[e];
    } else {
      const float hi = float(c[e]);
      f.c.f[e] = hi;
      if (a == Arith::DF) f.c.f[8 + e] = float(c[e] - double(hi));
    }
  }
}

// Kernel dispatch code of an encoded op (kind, conjugation, control form,
// register bit).
// Slot of the register-bit pair (a, b), a != b < 5 (see FFamily).
int pair_slot(int a, int b) {
  const int lo = std::min(a, b), hi = std::max(a, b);
  return lo * 4 - lo * (lo - 1) / 2 + (hi - lo - 1);
}

int dispatch_code(const FOp& f) {
  const bool c = f.conj != 0;
  const int S = kCodeSlots;
  switch (f.kind) {
    case FK_GEN: return (c ? FC_GEN_C : FC_GEN) * S + f.i0;
    case FK_H:  // uncontrolled; conj(H) = H
      if (f.flags & FF_SIDE) return FC_H_SIDE * S + f.i0 * 4 + f.i1;
      return FC_H * S + f.i0;
    case FK_SX:
      if (f.flags & FF_SIDE) return (c ? FC_SX_C_SIDE : FC_SX_SIDE) * S + f.i0 * 4 + f.i1;
      return (c ? FC_SX_C : FC_SX) * S + f.i0;
    case FK_SY:  // real
      if (f.flags & FF_SIDE) return FC_SY_SIDE * S + f.i0 * 4 + f.i1;
      return FC_SY * S + f.i0;
    case FK_X: return FC_X * S + f.i0;
    case FK_PHASE:
      if (f.rmask == 0) return FC_PHASE_ALL * S;
      if (popc(f.rmask) == 1) return FC_PHASE_BIT * S + __builtin_ctz(f.rmask);
      return FC_PHASE_MASK * S;
    case FK_SIGN: return FC_SIGN * S;
    case FK_SHEAR: return (f.i1 ? FC_SHEAR2 : FC_SHEAR) * S + f.i0;  // i1: the form
    case FK_PHASEU:
      if (f.rmask == 0) return FC_PHASEU_ALL * S;
      if (popc(f.rmask) == 1) return FC_PHASEU_BIT * S + __builtin_ctz(f.rmask);
      fail(QS_E_ARG, "fused planner: unscaled phase on several bits");
    case FK_MULI:
      if (f.rmask == 0) return FC_MULI_ALL * S;
      if (popc(f.rmask) == 1) return FC_MULI_BIT * S + __builtin_ctz(f.rmask);
      return FC_MULI_MASK * S;
    case FK_DEPH:
      if (f.asrc == BS_REG && f.bsrc == BS_REG) return FC_DEPH_PAIR * S + pair_slot(f.apos, f.bpos);
      return FC_DEPH * S;
    case FK_DEPOL: return FC_DEPOL * S + pair_slot(f.i0, f.i1);
    case FK_OFFPH: return FC_OFFPH * S + pair_slot(f.i0, f.i1);
    default: return FC_SCALE * S;
  }
}

// Device-side op encoding for one pass: stages of R register bits.  Stage op
// ranges are relative to the pass's first op.
void encode_pass(const Pass& p, int R, int k, Arith arith, std::vector<FOp>& fops,
                 std::vector<FStage>& fst) {
  const int32_t first = int32_t(fops.size());
  int lpos[64];
  for (int i = 0; i < 64; ++i) lpos[i] = -1;
  for (int i = 0; i < int(p.q.size()); ++i) lpos[p.q[i]] = i;
  // local positions of the tile qubits among x (bits outside the tile are
  // not local and are skipped)
  auto local_mask = [&](uint64_t x) {
    uint32_t m = 0;
    for (; x; x &= x - 1) {
      const int b = __builtin_ctzll(x);
      if (lpos[b] >= 0) m |= 1u << lpos[b];
    }
    return m;
  };

  // With FP64 (or double-float) arithmetic a stage boundary costs little
  // next to the arithmetic, while a phase on a bit that is not a register
  // bit runs on half-idle lanes; so there the bits a phase conditions on are
  // made register bits too.
  const bool phase_in_regs = arith != Arith::F32;
  auto needed = [&](const VOp& v) {
    uint32_t need = local_mask(v.xmask());
    if (phase_in_regs && (v.kind == FK_PHASE || v.kind == FK_PHASEU)) {
      const uint32_t c = local_mask(v.cond);
      if (popc(c) <= R) need |= c;
    }
    // a dephasing on two register bits runs over a compile-time half of the
    // register amplitudes
    if (v.kind == FK_DEPH) need |= local_mask(v.zmask());
    return need;
  };
  // Ops not yet in a stage, in pass order.  A stage takes them in order
  // while their needed bits fit in its R register bits; an op that does not
  // fit is deferred to a later stage, and a later op still joins this stage
  // if its bits fit and it commutes with every op deferred so far (no bit
  // either moves amplitudes along is a bit the other touches: the pass
  // builder's rule; against all deferred ops at once through the union of
  // their moved bits DX and of their touched bits DZ).  The ops of a stage
  // keep their pass order, and every op placed ahead of a deferred one
  // commutes with it: the result is that of the pass order.
  std::vector<size_t> rem(p.ops.size());
  for (size_t o = 0; o < rem.size(); ++o) rem[o] = o;
  // Per op: moved bits, touched bits, needed register positions.
  std::vector<uint64_t> ox(p.ops.size()), oz(p.ops.size());
  std::vector<uint32_t> oneed(p.ops.size());
  for (size_t o = 0; o < p.ops.size(); ++o) {
    ox[o] = p.ops[o].xmask();
    oz[o] = p.ops[o].zmask();
    oneed[o] = needed(p.ops[o]);
  }
  // One candidate register set: start from P0 and, with grow, add the bits
  // of each op that still fits; the ops taken, in pass order.
  auto simulate = [&](uint32_t P0, bool grow, uint32_t& P, std::vector<size_t>& take,
                      std::vector<size_t>& defer) {
    P = P0;
    take.clear();
    defer.clear();
    uint64_t DX = 0, DZ = 0;
    for (size_t o : rem) {
      const uint64_t xv = ox[o], zv = oz[o];
      if ((xv & (DX | DZ)) == 0 && (DX & (xv | zv)) == 0) {
        const uint32_t need = oneed[o];
        if ((need & ~P) == 0 || (grow && (take.empty() || popc(P | need) <= R))) {
          P |= need;
          take.push_back(o);
          continue;
        }
      }
      defer.push_back(o);
      DX |= xv;
      DZ |= zv;
    }
  };
  // The same scan over the first `limit` remaining ops only, counting the
  // moving ops (those needing register bits) it takes; -1 when it does not
  // take the first op (every stage must make progress).
  auto score = [&](uint32_t P0, bool grow, size_t limit) {
    uint32_t P = P0;
    uint64_t DX = 0, DZ = 0;
    int moved = 0;
    bool any = false;
    const size_t n = std::min(limit, rem.size());
    for (size_t i = 0; i < n; ++i) {
      const size_t o = rem[i];
      const uint64_t xv = ox[o], zv = oz[o];
      if ((xv & (DX | DZ)) == 0 && (DX & (xv | zv)) == 0) {
        const uint32_t need = oneed[o];
        if ((need & ~P) == 0 || (grow && (!any || popc(P | need) <= R))) {
          P |= need;
          any = true;
          moved += need != 0;
          continue;
        }
      }
      if (i == 0) return -1;
      DX |= xv;
      DZ |= zv;
    }
    return moved;
  };
  constexpr size_t kScoreOps = 128;
  std::vector<size_t> take, defer;
  while (!rem.empty()) {
    // Candidates: the in-order greedy set and every window of R adjacent
    // tile positions (on layered circuits a block of neighbouring qubits
    // can advance several layers in one stage, bounded by its neighbours,
    // where the first ops' bits are scattered across a layer).  Each is
    // scored on the next kScoreOps remaining ops by the moving ops it takes;
    // the highest wins (ties: the greedy set, then the lower window) and
    // only the winner scans every remaining op.
    uint32_t P0 = 0;
    bool grow = true;
    int best = score(0, true, kScoreOps);
    for (int w = 0; w + R <= k; ++w) {
      const uint32_t W = ((1u << R) - 1u) << w;
      const int m = score(W, false, kScoreOps);
      if (m > best) {
        best = m;
        P0 = W;
        grow = false;
      }
    }
    uint32_t P = 0;
    simulate(P0, grow, P, take, defer);
    rem.swap(defer);
    // spare register slots go first to the single bits the stage's phases
    // condition on (a phase on a lane bit runs on half-idle lanes), then to
    // the highest unused local bits (keeps low bits on lanes)
    for (size_t o : take) {
      if (popc(P) >= R) break;
      if (p.ops[o].kind == FK_PHASE || p.ops[o].kind == FK_PHASEU) {
        const uint32_t c = local_mask(p.ops[o].cond);
        if (popc(c) == 1) P |= c;
      }
    }
    for (int b = k - 1; b >= 0 && popc(P) < R; --b) P |= 1u << b;
    FStage st{};
    int idx[32];
    int n = 0;
    for (int b = 0; b < k; ++b)
      if ((P >> b) & 1) {
        idx[b] = n;
        st.pbits[n++] = uint8_t(b);
      }
    // the kernel reads exactly R distinct register positions below k
    if (n != R || (P >> k) != 0) fail(QS_E_ARG, "fused planner: stage register set is not R tile bits");
    st.op_begin = int32_t(fops.size()) - first;
    bool sign_seen = false;
    for (size_t o : take) {
      const VOp& v = p.ops[o];
      if (v.spread) {  // a copy made when the stage loads its amplitudes
        st.copy |= uint8_t(1u << idx[lpos[v.b0]]);
        continue;
      }
      FOp f{};
      f.kind = v.kind;
      f.conj = v.conj ? 1 : 0;
      if (v.kind <= FK_X || v.kind == FK_SHEAR || v.kind == FK_DEPOL || v.kind == FK_OFFPH)
        f.i0 = uint8_t(idx[lpos[v.b0]]);
      if (v.kind == FK_DEPOL || v.kind == FK_OFFPH) f.i1 = uint8_t(idx[lpos[v.b1]]);
      if (v.side >= 0) {
        f.i1 = uint8_t(idx[lpos[v.side]]);
        f.flags |= FF_SIDE;
      }
      if (v.kind == FK_SHEAR) f.i1 = v.c[1] != 0.0 ? 1 : 0;
      for (uint64_t cb = v.cond; cb; cb &= cb - 1) {
        const int b = __builtin_ctzll(cb);
        if (lpos[b] < 0) f.gmask |= uint64_t(1) << b;
        else if ((P >> lpos[b]) & 1) f.rmask |= uint8_t(1u << idx[lpos[b]]);
        else f.lmask |= 1u << lpos[b];
      }
      if (v.kind == FK_DEPH) {
        auto src = [&](int bit, uint8_t& s, uint8_t& pos) {
          if (lpos[bit] < 0) { s = BS_GLOBAL; pos = uint8_t(bit); }
          else if ((P >> lpos[bit]) & 1) { s = BS_REG; pos = uint8_t(idx[lpos[bit]]); }
          else { s = BS_LOCAL; pos = uint8_t(lpos[bit]); }
        };
        src(v.b0, f.asrc, f.apos);
        src(v.b1, f.bsrc, f.bpos);
      }
      set_coeffs(f, v.c, arith);
      if (v.kind == FK_OFFPH && f.i0 > f.i1) {  // c0 belongs to the lower register bit
        double c[8] = {v.c[1], v.c[0]};
        set_coeffs(f, c, arith);
      }
      if (v.kind == FK_PHASE || v.kind == FK_PHASEU || v.kind == FK_SIGN || v.kind == FK_MULI) {
        uint32_t touch = 0;  // register amplitudes j whose index has every rmask bit
        for (int j = 0; j < (1 << R); ++j)
          if ((uint32_t(j) & f.rmask) == f.rmask) touch |= 1u << j;
        f.c.u[15] = touch;
      }
      f.code = uint16_t(dispatch_code(f));
      if (f.lmask != 0 || f.gmask != 0) f.flags |= FF_COND;
      if (sign_seen && (v.kind <= FK_X || v.kind == FK_SHEAR || v.kind == FK_DEPOL)) f.flags |= FF_FLIP;
      if (v.kind == FK_DEPOL) f.flags |= FF_TWO;
      const bool deferred_sign = v.kind == FK_SIGN;
      if (deferred_sign) sign_seen = true;
      // consecutive pending sign flips under the same thread / tile condition
      // compose into one (the product of sign operators is their XOR)
      if (deferred_sign && int32_t(fops.size()) - first > st.op_begin) {
        FOp& prev = fops.back();
        if (prev.code == f.code && prev.lmask == f.lmask && prev.gmask == f.gmask) {
          prev.c.u[15] ^= f.c.u[15];
          continue;
        }
      }
      fops.push_back(f);
    }
    st.op_end = int32_t(fops.size()) - first;
    fst.push_back(st);
  }
}

double vop_flops(const VOp& v, int nq) {
  if (v.spread) return 0;
  const double dim = std::ldexp(1.0, nq), f = std::ldexp(1.0, -popc(v.cond));
  static const double pair_flops[5] = {28, 4, 4, 4, 0};  // H, sqrt(X), sqrt(Y) unscaled
  if (v.kind <= FK_X) return dim / 2 * f * pair_flops[v.kind];
  if (v.kind == FK_SHEAR) return dim / 2 * 8;
  if (v.kind == FK_PHASE) return dim * f * 6;
  if (v.kind == FK_PHASEU) return dim * f * 4;
  if (v.kind == FK_SCALE) return dim * 6;
  if (v.kind == FK_DEPH) return dim / 2 * 2;
  if (v.kind == FK_DEPOL) return dim / 4 * 8;
  if (v.kind == FK_OFFPH) return dim / 2 * 4;
  return 0;
}

// Arithmetic instructions (add, multiply, FMA: 1 each) one vector op issues,
// in the precision of the kernel's arithmetic.  Plain FP32/FP64 per pair:
// general 16, H / sqrt(X) / sqrt(Y) / shear 4; per touched amplitude: phase 4,
// dephasing 2; per quad: depolarising 4 (diagonal mix); per amplitude: scale 4.
// Double-float (packed: one instruction covers the real and imaginary
// parts): complex df add 11, multiply by a df factor 8, complex df product
// 27; in FP32-lane terms each packed instruction counts twice.
double vop_alu(const VOp& v, int nq, Arith a) {
  if (v.spread) return 0;
  const double dim = std::ldexp(1.0, nq), f = std::ldexp(1.0, -popc(v.cond));
  const bool d = a == Arith::DF;
  static const double plain_pair[5] = {16, 4, 4, 4, 0};
  static const double df_pair[5] = {2 * 130, 2 * 22, 2 * 22, 2 * 22, 0};
  if (v.kind <= FK_X) return dim / 2 * f * (d ? df_pair[v.kind] : plain_pair[v.kind]);
  if (v.kind == FK_SHEAR) return dim / 2 * (d ? 2 * 2 * (8 + 11) : 4);
  if (v.kind == FK_PHASE) return dim * f * (d ? 2 * 27 : 4);
  if (v.kind == FK_PHASEU) return dim * f * (d ? 2 * 27 : 2);
  if (v.kind == FK_SCALE) return dim * (d ? 2 * 27 : 4);
  if (v.kind == FK_DEPH) return dim / 2 * (d ? 2 * 8 : 2);
  if (v.kind == FK_DEPOL) return dim / 4 * (d ? 2 * 2 * (11 + 8) : 4);
  if (v.kind == FK_OFFPH) return dim / 2 * (d ? 2 * 27 : 2);
  return 0;
}

}  // namespace

void note_mixing(Reg& r, const GateOp& op) {
  uint64_t x = 0;
  switch (op.k) {
    case OpK::GEN: case OpK::H: case OpK::SX: case OpK::SY: case OpK::X: case OpK::DEPOL:
      x = uint64_t(1) << op.t;
      break;
    case OpK::MULTI:
      for (int i = 0; i < op.nt; ++i) x |= uint64_t(1) << op.tg[i];
      break;
    default:
      break;  // diagonal
  }
  if (r.density) x |= x << r.n;
  r.zero_bits &= ~x;
}

TileCfg tile_cfg(const Reg& r) {
  TileCfg c = r.prec == QS_C128 ? TileCfg{4, 12, 3} : TileCfg{5, 13, 4};
  // the env's "tile_low_qubits": fewer contiguous low qubits per tile leave
  // more tile qubits for the passes' windows, with shorter HBM chunks
  if (r.env && r.env->tile_low_qubits > 0) c.L = int(r.env->tile_low_qubits);
  return c;
}

bool fusable(const Reg& r) {
  const TileCfg c = tile_cfg(r);
  return r.nq >= c.R;  // a tile of 2^nq amplitudes worked by 2^(nq-R) threads
}

Arith arith_of(const Reg& r) {
  if (r.prec == QS_C64) return Arith::F32;
  return r.env->arith == 1 ? Arith::DF : Arith::F64;
}

void build_plan(const Reg& r, const std::vector<GateOp>& q, int k_req, uint64_t zero_in,
                std::complex<double> scale_in, RegPlan& out) {
  const Env& env = *r.env;
  TileCfg cfg = tile_cfg(r);
  // A register that fits one tile, in plain arithmetic, runs as one tile on
  // a thread-block cluster of up to "fused_cluster" CTAs (k_fused_cluster)
  // when the tile size is free or set to the register: 2^c CTAs of 4 warps,
  // i.e. R = k - 7 - c register bits (at least 2, at most the default), so
  // that 4c warps share the FP pipes of 4c SM sub-partitions instead of
  // 2^(k-R-5) warps on one SM.
  int cluster_c = 0;
  if (k_req == 0 && (env.tile_qubits == 0 || env.tile_qubits >= r.nq) && r.nq <= cfg.kmax &&
      arith_of(r) != Arith::DF && env.fused_cluster > 1) {
    int c = env.fused_cluster >= 8 ? 3 : env.fused_cluster >= 4 ? 2 : 1;
    const int Rc = std::max(2, std::min(cfg.R, r.nq - 7 - c));
    while (c > 0 && r.nq - Rc - 5 - c < 2) --c;
    if (c > 0) {
      cluster_c = c;
      cfg.R = Rc;
    }
  }
  int k = std::min(cfg.kmax, r.nq);
  if (cluster_c > 0) k = r.nq;
  else if (k_req > 0) k = std::min(k_req, r.nq);
  else if (env.tile_qubits > 0) k = std::min<int>(int(env.tile_qubits), r.nq);
  // a register of at most 18 qubits has too few tiles to fill the GPU: one
  // qubit less per tile doubles the tiles (SMs at work) for a few more
  // passes (measured, circuit of depth 20: complex128 12 / 16 / 18 qubits
  // 372-528 / 497 / 563 -> 283 / 369 / 405 us; complex64 16 / 18 qubits
  // 255 / 288 -> 232 / 265 us)
  else if (r.nq <= 18) k = std::min(k, cfg.kmax - 1);
  if (cluster_c == 0) {
    k = std::max(k, std::min(cfg.R + 5, r.nq));
    k = std::min(k, cfg.R + 8);  // at most 256 threads on one CTA
  }
  const int L = std::min(cfg.L, k);
  out = RegPlan{};
  out.k = k;
  out.L = L;
  out.R = cfg.R;
  out.cluster = cluster_c > 0 ? 1 << cluster_c : 0;
  out.arith = arith_of(r);

  std::vector<VOp> vops;
  vops.reserve(q.size() * 2);
  for (const GateOp& op : q) expand(r, op, vops);
  out.vops = int64_t(vops.size());
  uint64_t zero = zero_in;
  apply_zero_bits(vops, zero);
  out.zero_out = zero;
  merge_phases(vops, r.nq);
  absorb_into_general(vops);
  // FP64 defers factors down to 2^-500, so the first form (which passes a
  // phase's factor through, see unscale_phases) may take t up to 16
  decompose_general(vops, out.arith == Arith::F64 ? 16.0 : 1.0);
  merge_phases(vops, r.nq);
  if (out.arith != Arith::DF) unscale_phases(vops);
  // (side factors need R = 4 register slots: i0 * 4 + i1)
  if (r.density) scale_in *= defer_offdiag(vops, r.n, out.arith == Arith::F64 && cfg.R == 4);
  const int64_t cap = env.max_fused_ops > 0 ? std::min<int64_t>(env.max_fused_ops, kMaxPassOps)
                                            : kMaxPassOps;
  const std::vector<Pass> passes =
      plan(vops, r.nq, k, L, cap, out.arith == Arith::F64 ? 1000 : 80, scale_in, r.density ? r.n : 0);
  for (const Pass& p : passes) {
    FPass fp{};
    fp.k = k;
    fp.L = L;
    fp.nq = r.nq;
    fp.ntiles = int64_t(1) << (r.nq - k);
    fp.amps = r.d;
    for (int i = 0; i < k; ++i) fp.q[i] = uint8_t(p.q[i]);
    fp.stage_begin = int(out.fst.size());
    fp.op_begin = int(out.fops.size());
    encode_pass(p, cfg.R, k, out.arith, out.fops, out.fst);
    fp.stage_end = int(out.fst.size());
    fp.op_count = int(out.fops.size()) - fp.op_begin;
    out.fps.push_back(fp);
    double fl = 0;
    double al = 0;
    for (const VOp& v : p.ops) {
      fl += vop_flops(v, r.nq);
      al += vop_alu(v, r.nq, out.arith);
    }
    out.flops.push_back(fl);
    out.alu.push_back(al);
  }
}

}  // namespace qs
