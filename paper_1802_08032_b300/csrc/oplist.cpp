// Validation of gate arguments and conversion of bulk-call ops (QSOp) into
// the library's internal operations (host code, no device calls).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "runtime.h"

namespace qs {

void check_qubit(const Reg& r, int q, const char* what) {
  if (q < 0 || q >= r.n)
    fail(QS_E_QUBIT, std::string(what) + " qubit " + std::to_string(q) + " out of range [0, " +
                         std::to_string(r.n) + ")");
}

// Target plus controls: all in range and pairwise distinct.
uint64_t check_targets(const Reg& r, int target, const int* ctrls, int nc) {
  if (target >= 0) check_qubit(r, target, "target");
  uint64_t mask = 0;
  for (int k = 0; k < nc; ++k) {
    check_qubit(r, ctrls[k], "control");
    const uint64_t b = uint64_t(1) << ctrls[k];
    if ((mask & b) || ctrls[k] == target)
      fail(QS_E_DUP, "qubit " + std::to_string(ctrls[k]) + " repeated among target and controls");
    mask |= b;
  }
  return mask;
}

void check_unitary(const double* m) {
  // m: row-major u00 u01 u10 u11 as (re, im); max |U U^dagger - I| <= 1e-10.
  double worst = 0;
  for (int rr = 0; rr < 2; ++rr)
    for (int cc = 0; cc < 2; ++cc) {
      double re = 0, im = 0;
      for (int s = 0; s < 2; ++s) {
        const double ar = m[2 * (2 * rr + s)], ai = m[2 * (2 * rr + s) + 1];
        const double br = m[2 * (2 * cc + s)], bi = -m[2 * (2 * cc + s) + 1];
        re += ar * br - ai * bi;
        im += ar * bi + ai * br;
      }
      worst = std::max(worst, std::hypot(re - (rr == cc ? 1.0 : 0.0), im));
    }
  if (!(worst <= 1e-10)) fail(QS_E_UNITARY, "matrix is not unitary (max |UU^dagger - I| = " +
                                                std::to_string(worst) + ")");
}

GateOp make_op(OpK k, int t, uint64_t cmask) {
  GateOp op{};
  op.k = k;
  op.t = t;
  op.cmask = cmask;
  return op;
}

// Converts one bulk-call op into validated internal ops.
void convert_op(const Reg& r, const QSOp& o, std::vector<GateOp>& out) {
  const int nc = o.numControls;
  if (nc < 0 || nc > QS_MAX_OP_CONTROLS) fail(QS_E_ARG, "numControls out of range");
  switch (o.kind) {
    case QS_OP_H: check_qubit(r, o.target, "target"); out.push_back(make_op(OpK::H, o.target, 0)); return;
    case QS_OP_X: check_qubit(r, o.target, "target"); out.push_back(make_op(OpK::X, o.target, 0)); return;
    case QS_OP_SQRTX: check_qubit(r, o.target, "target"); out.push_back(make_op(OpK::SX, o.target, 0)); return;
    case QS_OP_SQRTY: check_qubit(r, o.target, "target"); out.push_back(make_op(OpK::SY, o.target, 0)); return;
    case QS_OP_T:
    case QS_OP_PHASE: {
      check_qubit(r, o.target, "target");
      const double ang = o.kind == QS_OP_T ? M_PI / 4 : o.params[0];
      GateOp op = make_op(OpK::PHASE, o.target, 0);
      op.m[0] = o.kind == QS_OP_T ? std::sqrt(0.5) : std::cos(ang);
      op.m[1] = o.kind == QS_OP_T ? std::sqrt(0.5) : std::sin(ang);
      out.push_back(op);
      return;
    }
    case QS_OP_COMPACT: {
      check_qubit(r, o.target, "target");
      const double ar = o.params[0], ai = o.params[1], br = o.params[2], bi = o.params[3];
      const double nrm = ar * ar + ai * ai + br * br + bi * bi;
      if (!(std::fabs(nrm - 1.0) <= 1e-10))
        fail(QS_E_UNITARY, "compactUnitary: |alpha|^2 + |beta|^2 = " + std::to_string(nrm));
      GateOp op = make_op(OpK::GEN, o.target, 0);
      // [[alpha, -conj(beta)], [beta, conj(alpha)]]
      const double m[8] = {ar, ai, -br, bi, br, bi, ar, -ai};
      std::memcpy(op.m, m, sizeof(m));
      out.push_back(op);
      return;
    }
    case QS_OP_UNITARY:
    case QS_OP_CUNITARY:
    case QS_OP_CNOT: {
      const int ncu = o.kind == QS_OP_UNITARY ? 0 : (o.kind == QS_OP_CNOT ? 1 : nc);
      if (o.kind == QS_OP_CNOT && nc != 1 && nc != 0) fail(QS_E_ARG, "CNOT takes one control");
      const uint64_t cm = check_targets(r, o.target, o.controls, ncu);
      if (o.kind == QS_OP_CNOT) {
        out.push_back(make_op(OpK::X, o.target, cm));
        return;
      }
      check_unitary(o.params);
      GateOp op = make_op(OpK::GEN, o.target, cm);
      std::memcpy(op.m, o.params, sizeof(op.m));
      out.push_back(op);
      return;
    }
    case QS_OP_CZ: {
      const int c[1] = {o.target2};
      const uint64_t cm = check_targets(r, o.target, c, 1);
      out.push_back(make_op(OpK::SIGN, -1, cm | (uint64_t(1) << o.target)));
      return;
    }
    case QS_OP_MCPF: {
      if (nc < 1) fail(QS_E_ARG, "multiControlledPhaseFlip needs at least one qubit");
      const uint64_t cm = check_targets(r, -1, o.controls, nc);
      out.push_back(make_op(OpK::SIGN, -1, cm));
      return;
    }
    case QS_OP_DEPHASE:
    case QS_OP_DEPOL: {
      if (!r.density) fail(QS_E_NOT_DENSITY, "noise channel on a state vector");
      check_qubit(r, o.target, "target");
      const double p = o.params[0];
      const double pmax = o.kind == QS_OP_DEPHASE ? 0.5 : 0.75;
      if (!(p >= 0.0 && p <= pmax))
        fail(QS_E_PROB, "channel probability " + std::to_string(p) + " outside [0, " +
                            std::to_string(pmax) + "]");
      GateOp op = make_op(o.kind == QS_OP_DEPHASE ? OpK::DEPHASE : OpK::DEPOL, o.target, 0);
      op.m[0] = p;
      out.push_back(op);
      return;
    }
    default: fail(QS_E_ARG, "unknown op kind " + std::to_string(o.kind));
  }
}

void convert_ops(const Reg& r, const QSOp* ops, int64_t n, std::vector<GateOp>& out) {
  for (int64_t i = 0; i < n; ++i) {
    try {
      convert_op(r, ops[i], out);
    } catch (Error& e) {
      e.msg = "op " + std::to_string(i) + ": " + e.msg;
      throw;
    }
  }
}

}  // namespace qs
