// Encoding of fused-pass operations, shared by the host planner and the
// fused tile kernel (plain C++: no device code).
#pragma once
#ifndef __CUDACC_RTC__
#include <cstdint>
#endif

namespace qs {

// Vector-level operations of the fused engine.
enum FKind : uint8_t {
  FK_GEN = 0, FK_H = 1, FK_SX = 2, FK_SY = 3, FK_X = 4,   // pair ops (PairKind order)
  FK_PHASE = 5,   // multiply by (c0, c1) where the condition holds
  FK_SIGN = 6,    // negate where the condition holds
  FK_DEPH = 7,    // scale by c0 where bit A != bit B
  FK_DEPOL = 8,   // depolarising quad on register bits (i0 = row bit, i1 = column bit):
                  // the diagonal pair only, (x, y) -> (x + r y, y + r x), r = c0 (the
                  // off-diagonal factor and the common factor 1 - m are deferred, see
                  // the planner)
  FK_SCALE = 9,   // multiply every amplitude by the complex (c0, c1)
  FK_MULI = 10,   // multiply by i where the condition holds (no arithmetic)
  FK_SHEAR = 11,  // pair op: (x, y) -> (x - t y, y + u x), or (t x - y, x + t y): a real
                  // rotation up to a factor deferred like the dropped ones (c0 = t, c4 = u;
                  // u = t unless a phase's factor passes through, see the planner)
  FK_PHASEU = 12,  // multiply by (1 + i t) where the condition holds (c0 = t): a phase
                   // whose real factor the next pair update on its bit applies
  FK_OFFPH = 13    // density-matrix phase pair on register bits i0 < i1: multiply by
                   // (1 + i c0) where bit i0 = 1, bit i1 = 0 and by (1 + i c1) where
                   // bit i0 = 0, bit i1 = 1 (a row phase and its conjugate column
                   // phase; the real factor is deferred with the off-diagonal ones)
};
// H, sqrt(X) and sqrt(Y) carry one coefficient, c0: a real factor applied to
// their bit-1 input y (1 unless a preceding FK_PHASEU on the bit left its
// real factor to them).
// In this engine H, sqrt(X) and sqrt(Y) are applied WITHOUT their scalar
// factors: H = (1/sqrt 2) [[1, 1], [1, -1]], sqrt(X) = ((1+i)/2) [[1, -i], [-i, 1]],
// sqrt(Y) = ((1+i)/2) [[1, -1], [1, 1]]; the bracketed matrices need additions
// only.  Those gates are uncontrolled, so the dropped factors multiply the
// whole vector; the planner emits an FK_SCALE with their accumulated complex
// product in the last pass of a plan (every op is linear, so the factor
// commutes with all of them), and earlier if the growth would leave the
// arithmetic's exponent range.  The conjugated forms (density-matrix column
// updates) drop the conjugate factors: [[1, i], [i, 1]] and (1-i)/2.

// Where a single bit of the amplitude index comes from, within a stage.
enum BitSrc : uint8_t { BS_REG = 0, BS_LOCAL = 1, BS_GLOBAL = 2 };

// Kernel dispatch of an operation: code = family * 16 + slot, where the slot
// is the target register bit, or the index of a register-bit pair (a, b),
// a < b, in the order (0,1) (0,2) (0,3) (0,4) (1,2) (1,3) (1,4) (2,3) (2,4)
// (3,4); so kind, conjugation and bits come from one word.  The general
// matrix and X test register-bit controls per pair (compiling uncontrolled
// copies of them as well costs the kernel registers it does not have).
// Sign flips only update a pending mask (see process_tile).
enum FFamily : uint8_t {
  FC_GEN = 0, FC_GEN_C = 1, FC_H = 2, FC_SX = 3, FC_SX_C = 4, FC_SY = 5, FC_X = 6,
  FC_PHASE_BIT = 7, FC_PHASE_ALL = 8, FC_PHASE_MASK = 9,
  FC_SIGN = 10, FC_DEPH = 11, FC_DEPOL = 12, FC_SCALE = 13,
  FC_MULI_BIT = 14, FC_MULI_ALL = 15, FC_MULI_MASK = 16,
  FC_SHEAR = 17, FC_SHEAR2 = 18,  // (x - t y, y + t x); (t x - y, x + t y)
  FC_PHASEU_BIT = 19, FC_PHASEU_ALL = 20,
  FC_DEPH_PAIR = 21,  // FK_DEPH whose two bits are register bits (pair slot)
  FC_OFFPH = 22,      // pair slot
  // H, sqrt(X), conjugated sqrt(X), sqrt(Y) on register bit i0 with the real
  // factor c0 on the input whose register bit i1 differs from its bit i0
  // (FP64 arithmetic, R = 4 only; slot = i0 * 4 + i1)
  FC_H_SIDE = 23, FC_SX_SIDE = 24, FC_SX_C_SIDE = 25, FC_SY_SIDE = 26
};
constexpr int kCodeSlots = 16;
// FOp::flags
enum : uint8_t {
  FF_COND = 1,  // lmask or gmask set: a per-thread / per-tile predicate
  FF_FLIP = 2,  // a sign flip precedes the op in its stage: check pending flips
  FF_TWO = 4,   // the op moves amplitudes along register bits i0 and i1
  FF_SIDE = 8   // H / sqrt(X) / sqrt(Y) with the side factor on register bit i1 (encoding only)
};

// One operation as applied in one stage (all masks pre-split by the host).
// Coefficients (matrix re/im row-major; PHASE cos, sin; DEPH factor; DEPOL
// keep, move, off; SCALE factor) are stored in the form the kernel's
// arithmetic uses: doubles (FP64), floats (FP32), or float pairs hi[0..7]
// lo[8..15] (double-float).
struct FOp {
  uint8_t kind;
  uint8_t conj;     // pair ops: apply conj(G)
  uint8_t i0, i1;   // register-bit indices (pair target; DEPOL row/column)
  uint8_t asrc, apos, bsrc, bpos;  // DEPH bit sources
  uint16_t code;    // FFamily * kCodeSlots + slot
  uint8_t flags;    // FF_*
  uint8_t rmask;    // condition bits among the register bits (bit i = register bit i)
  uint32_t lmask;   // condition bits among the other local bits (local positions)
  uint64_t gmask;   // condition bits outside the tile (global positions)
  union {
    double d[8];
    float f[16];
    uint32_t u[16];  // PHASE / SIGN / MULI: u[15] = the register amplitudes j the op touches
  } c;
};
static_assert(sizeof(FOp) == 88, "FOp layout");

struct FStage {
  uint8_t pbits[7];          // local positions of the register bits (R used)
  // Register bits whose bit-1 amplitudes are loaded as copies of the bit-0
  // ones: an H / sqrt(X) / sqrt(Y) on a bit whose bit-1 amplitudes are all
  // 0 maps (x, 0) to (x, x) (unscaled; sqrt(X) then multiplies the copy by
  // -i or i, as separate ops).  Every op of the stage before it leaves that
  // bit alone, so the copy can be made when the stage loads its amplitudes.
  uint8_t copy;
  int32_t op_begin, op_end;  // relative to the pass's first op
};

struct FPass {
  int k, L, nq;
  int stage_begin, stage_end;  // indices into the stage array
  int op_begin, op_count;      // the pass's ops in the op array
  int init;                    // 1: the register starts in |0...0> (tiles are generated, not loaded)
  int pad_;
  int64_t ntiles;
  void* amps;                  // register amplitudes (batched launches; null = kernel argument)
  uint8_t q[24];               // tile qubits, ascending; q[i] = i for i < L
};

static_assert(sizeof(FPass) % 8 == 0 && sizeof(FPass) / 8 <= 256, "FPass word copy");

// One unit of a batched launch: tile `tile` of pass `pass`.
struct BItem {
  int32_t pass;
  int32_t pad_;
  int64_t tile;
};

constexpr int kMaxPassOps = 256;

}  // namespace qs
