// Host-side check of the fused-pass planner (test infrastructure; built by
// tests/test_planner.py with the host compiler against the library's
// planner.cpp and oplist.cpp, no GPU involved).
//
// Reads QSOp records from stdin, plans them for a register of the given
// shape and checks the invariants the fused tile kernel relies on.  With
// emulate = 1 it then applies the encoded passes to |0...0> on the CPU,
// following what each encoded operation means (tile gather, register
// stages, per-thread and per-tile conditions, pending sign flips), and
// writes the final 2^nq amplitudes (re, im doubles) to stdout after a line
// "STATE".  The test compares that state with the oracle.
//
// usage: planner_check n density prec arith k_req emulate [fresh [tile_low_qubits]]
#include <algorithm>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "plan.h"
#include "runtime.h"

using namespace qs;
using cd = std::complex<double>;

static int violations = 0;
#define CHECK(cond, ...)                   \
  do {                                     \
    if (!(cond)) {                         \
      ++violations;                        \
      if (violations <= 20) {              \
        std::fprintf(stderr, __VA_ARGS__); \
        std::fprintf(stderr, "\n");        \
      }                                    \
    }                                      \
  } while (0)

static int popc64(uint64_t x) { return __builtin_popcountll(x); }

// Register-bit pair of a pair slot (the order of the FFamily comment).
static void slot_pair(int s, int& a, int& b) {
  static const int A[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3}, B[10] = {1, 2, 3, 4, 2, 3, 4, 3, 4, 4};
  a = A[s];
  b = B[s];
}

static double coef(const FOp& f, int e, Arith a) {
  if (a == Arith::F64) return f.c.d[e];
  if (a == Arith::F32) return double(f.c.f[e]);
  return double(f.c.f[e]) + double(f.c.f[8 + e]);
}

static void check_plan(const RegPlan& pl, int nq) {
  const int R = pl.R, k = pl.k, L = pl.L;
  CHECK(R >= 1 && R <= 5 && k >= R && k <= nq, "bad k %d / R %d", k, R);
  for (size_t pi = 0; pi < pl.fps.size(); ++pi) {
    const FPass& P = pl.fps[pi];
    CHECK(P.k == k && P.L == L && P.nq == nq, "pass %zu: shape", pi);
    CHECK(P.ntiles == (int64_t(1) << (nq - k)), "pass %zu: ntiles", pi);
    uint64_t tile = 0;
    for (int i = 0; i < k; ++i) {
      CHECK(P.q[i] < nq, "pass %zu: tile qubit %d out of range", pi, P.q[i]);
      if (i < L) CHECK(P.q[i] == i, "pass %zu: low qubit %d", pi, i);
      if (i > 0) CHECK(P.q[i] > P.q[i - 1], "pass %zu: tile qubits not ascending", pi);
      tile |= uint64_t(1) << P.q[i];
    }
    CHECK(P.stage_end > P.stage_begin, "pass %zu: no stage", pi);
    int next = 0;
    for (int s = P.stage_begin; s < P.stage_end; ++s) {
      const FStage& st = pl.fst[s];
      CHECK(st.op_begin == next && st.op_end >= st.op_begin, "pass %zu stage %d: op range", pi, s);
      next = st.op_end;
      uint32_t pm = 0;
      CHECK((st.copy >> R) == 0, "pass %zu stage %d: copy bits", pi, s);
      for (int i = 0; i < R; ++i) {
        CHECK(st.pbits[i] < k, "pass %zu stage %d: register position %d >= k", pi, s, st.pbits[i]);
        if (i > 0) CHECK(st.pbits[i] > st.pbits[i - 1], "pass %zu stage %d: positions not ascending", pi, s);
        pm |= 1u << st.pbits[i];
      }
      for (int o = st.op_begin; o < st.op_end; ++o) {
        const FOp& f = pl.fops[P.op_begin + o];
        const int fam = f.code / kCodeSlots, slot = f.code % kCodeSlots;
        CHECK(fam <= FC_SY_SIDE, "op %d: family %d", o, fam);
        if (fam >= FC_H_SIDE && fam <= FC_SY_SIDE)
          CHECK(R == 4 && slot / 4 != slot % 4 && f.i0 == slot / 4 && f.i1 == slot % 4 && f.rmask == 0 &&
                    f.lmask == 0 && f.gmask == 0 && ((f.flags & FF_SIDE) != 0),
                "op %d: side-factor pair update", o);
        CHECK(f.rmask < (1u << R), "op %d: rmask", o);
        CHECK((f.lmask & pm) == 0 && (f.lmask >> k) == 0, "op %d: lmask on a register / non-tile bit", o);
        CHECK((f.gmask & tile) == 0 && (nq == 64 || (f.gmask >> nq) == 0), "op %d: gmask inside the tile", o);
        CHECK(((f.flags & FF_COND) != 0) == (f.lmask != 0 || f.gmask != 0), "op %d: FF_COND", o);
        if (fam <= FC_X || fam == FC_PHASE_BIT || fam == FC_MULI_BIT || fam == FC_SHEAR || fam == FC_SHEAR2 ||
            fam == FC_PHASEU_BIT)
          CHECK(slot < R, "op %d: slot %d >= R", o, slot);
        if (fam == FC_SHEAR || fam == FC_SHEAR2)
          CHECK(f.rmask == 0 && f.lmask == 0 && f.gmask == 0 && f.i0 == slot, "op %d: shear", o);
        if (fam <= FC_X) {
          CHECK(f.i0 == slot && ((f.rmask >> f.i0) & 1u) == 0, "op %d: pair target", o);
          if (fam != FC_GEN && fam != FC_GEN_C && fam != FC_X) CHECK(f.rmask == 0, "op %d: controlled add-only pair", o);
        }
        if (fam == FC_PHASE_BIT) CHECK(popc64(f.rmask) == 1 && (f.rmask >> slot) == 1u, "op %d: phase bit", o);
        if (fam == FC_PHASE_ALL || fam == FC_MULI_ALL) CHECK(f.rmask == 0, "op %d: phase all", o);
        if (fam == FC_MULI_BIT) CHECK(popc64(f.rmask) == 1 && (f.rmask >> slot) == 1u, "op %d: i bit", o);
        if (fam == FC_DEPOL) {
          int a, b;
          slot_pair(slot, a, b);
          CHECK(b < R && std::min<int>(f.i0, f.i1) == a && std::max<int>(f.i0, f.i1) == b, "op %d: depol bits", o);
        }
        if (fam == FC_DEPH_PAIR) {
          int a, b;
          slot_pair(slot, a, b);
          CHECK(b < R && f.asrc == BS_REG && f.bsrc == BS_REG &&
                    std::min<int>(f.apos, f.bpos) == a && std::max<int>(f.apos, f.bpos) == b,
                "op %d: dephasing register bits", o);
        }
        if (fam == FC_DEPH) CHECK(f.asrc != BS_REG || f.bsrc != BS_REG, "op %d: dephasing form", o);
        if (fam == FC_OFFPH) {
          int a, b;
          slot_pair(slot, a, b);
          CHECK(b < R && std::min<int>(f.i0, f.i1) == a && std::max<int>(f.i0, f.i1) == b && f.rmask == 0 &&
                    f.lmask == 0 && f.gmask == 0,
                "op %d: row / column phase bits", o);
        }
      }
    }
    CHECK(next == P.op_count, "pass %zu: stages cover %d of %d ops", pi, next, P.op_count);
  }
}

// |0...0> through the encoded passes.
static std::vector<cd> emulate(const RegPlan& pl, int nq) {
  std::vector<cd> psi(size_t(1) << nq, cd(0, 0));
  psi[0] = 1.0;
  const int R = pl.R, k = pl.k;
  for (const FPass& P : pl.fps) {
    for (int64_t tau = 0; tau < P.ntiles; ++tau) {
      // the tile's global base: tau's bits over the non-tile positions
      uint64_t base = 0;
      int bit = 0;
      uint64_t tile = 0;
      for (int i = 0; i < k; ++i) tile |= uint64_t(1) << P.q[i];
      for (int g = 0; g < nq; ++g)
        if (!((tile >> g) & 1)) base |= uint64_t((tau >> bit++) & 1) << g;
      auto gidx = [&](uint32_t l) {
        uint64_t x = base;
        for (int i = 0; i < k; ++i) x |= uint64_t((l >> i) & 1u) << P.q[i];
        return x;
      };
      std::vector<cd> t(size_t(1) << k);
      for (uint32_t l = 0; l < t.size(); ++l) t[l] = psi[gidx(l)];
      for (int s = P.stage_begin; s < P.stage_end; ++s) {
        const FStage& st = pl.fst[s];
        for (uint32_t th = 0; th < (1u << (k - R)); ++th) {
          // this thread's local index: th spread over the non-register positions
          uint32_t tl = 0;
          int tb = 0;
          uint32_t pm = 0;
          for (int i = 0; i < R; ++i) pm |= 1u << st.pbits[i];
          for (int p = 0; p < k; ++p)
            if (!((pm >> p) & 1)) tl |= ((th >> tb++) & 1u) << p;
          auto loc = [&](int j) {
            uint32_t x = tl;
            for (int i = 0; i < R; ++i)
              if ((j >> i) & 1) x |= 1u << st.pbits[i];
            return x;
          };
          const int nj = 1 << R;
          cd v[32];
          // copy bits: their bit-1 amplitudes start as the bit-0 ones (the
          // planner's claim that the bit-1 ones are 0 is not used: overwritten)
          for (int j = 0; j < nj; ++j) v[j] = t[loc(j & ~int(st.copy))];
          uint32_t flips = 0;
          auto flush_flips = [&] {
            for (int j = 0; j < nj; ++j)
              if ((flips >> j) & 1u) v[j] = -v[j];
            flips = 0;
          };
          for (int o = st.op_begin; o < st.op_end; ++o) {
            const FOp& f = pl.fops[P.op_begin + o];
            if ((tl & f.lmask) != f.lmask || (base & f.gmask) != f.gmask) continue;
            const int fam = f.code / kCodeSlots, slot = f.code % kCodeSlots;
            if (fam == FC_SIGN) {
              flips ^= f.c.u[15];
              continue;
            }
            const bool side = fam >= FC_H_SIDE && fam <= FC_SY_SIDE;
            if (fam <= FC_X || fam == FC_DEPOL || fam == FC_SHEAR || fam == FC_SHEAR2 || side) flush_flips();
            auto c = [&](int e) { return coef(f, e, pl.arith); };
            if (fam <= FC_X) {
              const int I = slot;
              cd g00(1, 0), g01(0, 0), g10(0, 0), g11(1, 0);
              if (fam == FC_GEN || fam == FC_GEN_C) {
                g00 = cd(c(0), c(1)); g01 = cd(c(2), c(3)); g10 = cd(c(4), c(5)); g11 = cd(c(6), c(7));
                if (fam == FC_GEN_C) { g00 = std::conj(g00); g01 = std::conj(g01); g10 = std::conj(g10); g11 = std::conj(g11); }
              } else if (fam == FC_H) { g01 = 1; g10 = 1; g11 = -1; }
              else if (fam == FC_SX) { g01 = cd(0, -1); g10 = cd(0, -1); }
              else if (fam == FC_SX_C) { g01 = cd(0, 1); g10 = cd(0, 1); }
              else if (fam == FC_SY) { g01 = -1; g10 = 1; }
              else { g00 = 0; g01 = 1; g10 = 1; g11 = 0; }  // X
              if (fam >= FC_H && fam <= FC_SY) {  // c0: factor on the bit-1 input
                g01 *= c(0);
                g11 *= c(0);
              }
              for (int j = 0; j < nj; ++j) {
                if ((j >> I) & 1) continue;
                if ((uint32_t(j) & f.rmask) != f.rmask) continue;
                const cd x = v[j], y = v[j | (1 << I)];
                v[j] = g00 * x + g01 * y;
                v[j | (1 << I)] = g10 * x + g11 * y;
              }
            } else if (fam == FC_PHASE_BIT || fam == FC_PHASE_ALL || fam == FC_PHASE_MASK || fam == FC_SCALE) {
              const cd ph(c(0), c(1));
              for (int j = 0; j < nj; ++j) {
                bool touch = true;
                if (fam == FC_PHASE_BIT) touch = (j >> slot) & 1;
                if (fam == FC_PHASE_MASK) touch = (f.c.u[15] >> j) & 1u;
                if (touch) v[j] *= ph;
              }
            } else if (fam == FC_PHASEU_BIT || fam == FC_PHASEU_ALL) {
              const cd u(1.0, c(0));
              for (int j = 0; j < nj; ++j)
                if (fam == FC_PHASEU_ALL || ((j >> slot) & 1)) v[j] *= u;
            } else if (fam == FC_SHEAR || fam == FC_SHEAR2) {
              const double t = c(0);
              for (int j = 0; j < nj; ++j) {
                if ((j >> slot) & 1) continue;
                const cd x = v[j], y = v[j | (1 << slot)];
                v[j] = fam == FC_SHEAR ? x - t * y : t * x - y;
                v[j | (1 << slot)] = fam == FC_SHEAR ? y + c(4) * x : x + t * y;
              }
            } else if (fam == FC_MULI_BIT || fam == FC_MULI_ALL || fam == FC_MULI_MASK) {
              for (int j = 0; j < nj; ++j) {
                bool touch = true;
                if (fam == FC_MULI_BIT) touch = (j >> slot) & 1;
                if (fam == FC_MULI_MASK) touch = (f.c.u[15] >> j) & 1u;
                if (touch) v[j] *= cd(0, 1);
              }
            } else if (fam == FC_DEPH) {
              auto bv = [&](uint8_t src, uint8_t pos, int j) -> int {
                if (src == BS_REG) return (j >> pos) & 1;
                if (src == BS_LOCAL) return int((tl >> pos) & 1u);
                return int((base >> pos) & 1u);
              };
              for (int j = 0; j < nj; ++j)
                if (bv(f.asrc, f.apos, j) != bv(f.bsrc, f.bpos, j)) v[j] *= c(0);
            } else if (side) {  // unscaled H / sqrt(X) / sqrt(Y) on bit I, c0 on the input whose bit J != bit I
              const int I = slot / 4, J = slot % 4;
              cd g01(1, 0), g10(1, 0), g11(-1, 0);  // H
              if (fam == FC_SX_SIDE) { g01 = cd(0, -1); g10 = cd(0, -1); g11 = 1; }
              if (fam == FC_SX_C_SIDE) { g01 = cd(0, 1); g10 = cd(0, 1); g11 = 1; }
              if (fam == FC_SY_SIDE) { g01 = -1; g10 = 1; g11 = 1; }
              for (int j = 0; j < nj; ++j) {
                if ((j >> I) & 1) continue;
                cd x = v[j], y = v[j | (1 << I)];
                if ((j >> J) & 1) x *= c(0);
                else y *= c(0);
                v[j] = x + g01 * y;
                v[j | (1 << I)] = g10 * x + g11 * y;
              }
            } else if (fam == FC_OFFPH) {  // (1 + i c0) where only bit a is set, (1 + i c1) only b
              int a, b;
              slot_pair(slot, a, b);
              for (int j = 0; j < nj; ++j) {
                const int lo = (j >> a) & 1, hi = (j >> b) & 1;
                if (lo && !hi) v[j] *= cd(1.0, c(0));
                if (!lo && hi) v[j] *= cd(1.0, c(1));
              }
            } else if (fam == FC_DEPH_PAIR) {
              int a, b;
              slot_pair(slot, a, b);
              for (int j = 0; j < nj; ++j)
                if (((j >> a) ^ (j >> b)) & 1) v[j] *= c(0);
            } else if (fam == FC_DEPOL) {  // the diagonal pair only: (x + r y, y + r x)
              int a, b;
              slot_pair(slot, a, b);
              for (int j = 0; j < nj; ++j) {
                if ((j >> a) & 1 || (j >> b) & 1) continue;
                const int jd = j | (1 << a) | (1 << b);
                const cd d0 = v[j], d1 = v[jd];
                v[j] = d0 + c(0) * d1;
                v[jd] = d1 + c(0) * d0;
              }
            }
          }
          flush_flips();
          for (int j = 0; j < nj; ++j) t[loc(j)] = v[j];
        }
      }
      for (uint32_t l = 0; l < t.size(); ++l) psi[gidx(l)] = t[l];
    }
  }
  return psi;
}

int main(int argc, char** argv) {
  if (argc < 7) {
    std::fprintf(stderr, "usage: planner_check n density prec arith k_req emulate\n");
    return 2;
  }
  const int n = std::atoi(argv[1]), density = std::atoi(argv[2]), prec = std::atoi(argv[3]);
  const int arith = std::atoi(argv[4]), k_req = std::atoi(argv[5]), emu = std::atoi(argv[6]);
  const int fresh = argc > 7 ? std::atoi(argv[7]) : 1;
  const int tile_low = argc > 8 ? std::atoi(argv[8]) : 0;
  Env env;
  env.arith = arith;
  env.tile_low_qubits = tile_low;
  Reg r;
  r.env = &env;
  r.n = n;
  r.density = density != 0;
  r.nq = density ? 2 * n : n;
  r.prec = prec;
  r.dim = int64_t(1) << r.nq;
  std::vector<QSOp> ops;
  QSOp o;
  while (std::fread(&o, sizeof(o), 1, stdin) == 1) ops.push_back(o);
  RegPlan pl;
  try {
    std::vector<GateOp> g;
    convert_ops(r, ops.data(), int64_t(ops.size()), g);
    // a zeroed register unless told otherwise (argument 7 = 0)
    build_plan(r, g, k_req, fresh ? (uint64_t(1) << r.nq) - 1 : 0, 1.0, pl);
  } catch (const Error& e) {
    std::printf("ERROR %d %s\n", e.code, e.msg.c_str());
    return 1;
  }
  check_plan(pl, r.nq);
  std::printf("PLAN passes %zu stages %zu ops %zu k %d R %d violations %d\n", pl.fps.size(),
              pl.fst.size(), pl.fops.size(), pl.k, pl.R, violations);
  if (emu && violations == 0) {
    const std::vector<cd> psi = emulate(pl, r.nq);
    std::printf("STATE\n");
    std::fflush(stdout);
    std::fwrite(psi.data(), sizeof(cd), psi.size(), stdout);
  }
  return violations ? 3 : 0;
}
