// Schedule planner of partitioned state vectors (host only; see
// partition.h).  The executor is partition.cu.
#include "partition.h"

#include <algorithm>
#include <complex>
#include <limits>
#include <string>

namespace qs {

namespace {

// The qubit an op moves amplitudes along, or -1 for a diagonal op.
int moved_qubit(const GateOp& op) {
  switch (op.k) {
    case OpK::GEN:
    case OpK::H:
    case OpK::SX:
    case OpK::SY:
    case OpK::X:
      return op.t;
    case OpK::PHASE:
    case OpK::SIGN:
      return -1;
    default:
      fail(QS_E_ARG, "partitioned registers take single-target gates, phases and sign flips only");
  }
}

}  // namespace

std::vector<PartStep> plan_partition(int n, int m, const std::vector<GateOp>& ops, std::vector<int>& perm) {
  if (m < 1 || m > n) fail(QS_E_ARG, "a partitioned register needs 1 <= local qubits <= qubits");
  if (int(perm.size()) != n) fail(QS_E_ARG, "qubit map of the wrong size");
  // logical qubit at each physical position
  std::vector<int> at(size_t(n), -1);
  for (int q = 0; q < n; ++q) at[size_t(perm[size_t(q)])] = q;
  std::vector<int> moved(ops.size());
  for (size_t i = 0; i < ops.size(); ++i) moved[i] = moved_qubit(ops[i]);
  std::vector<PartStep> steps;
  for (size_t i = 0; i < ops.size(); ++i) {
    const int q = moved[i];
    if (q >= 0 && perm[size_t(q)] >= m) {
      // next use (as a moved qubit) of every local position's qubit
      int victim = -1;
      size_t best = 0;
      for (int l = 0; l < m; ++l) {
        const int lq = at[size_t(l)];
        size_t next = std::numeric_limits<size_t>::max();
        for (size_t j = i; j < ops.size(); ++j)
          if (moved[j] == lq) {
            next = j;
            break;
          }
        if (victim < 0 || next > best) {
          victim = l;
          best = next;
        }
      }
      const int g = perm[size_t(q)];
      steps.push_back(PartStep{PartStep::SWAP, -1, g, victim});
      const int vq = at[size_t(victim)];
      perm[size_t(q)] = victim;
      perm[size_t(vq)] = g;
      at[size_t(victim)] = q;
      at[size_t(g)] = vq;
    }
    steps.push_back(PartStep{PartStep::LOCAL, int32_t(i), -1, -1});
  }
  return steps;
}

bool part_gate(const GateOp& op, const std::vector<int>& perm, int m, int64_t part, GateOp& out, bool& has_op,
               std::complex<double>& scalar) {
  has_op = false;
  scalar = 1.0;
  auto global_bit = [&](int phys) { return int((part >> (phys - m)) & 1); };
  // controls (or the flipped set of a sign flip), mapped; global bits must
  // all be 1 for this part, the local ones stay
  uint64_t local = 0;
  for (int q = 0; q < 64; ++q) {
    if (!((op.cmask >> q) & 1u)) continue;
    const int p = perm[size_t(q)];
    if (p >= m) {
      if (!global_bit(p)) return false;
    } else {
      local |= uint64_t(1) << p;
    }
  }
  out = op;
  out.cmask = local;
  if (op.k == OpK::SIGN) {
    if (local) has_op = true;
    else scalar = -1.0;  // every flipped qubit global and set: the whole part
    return true;
  }
  const int pt = perm[size_t(op.t)];
  if (op.k == OpK::PHASE && pt >= m) {
    // a phase on a global qubit: the whole part when its bit is 1
    if (!global_bit(pt)) return false;
    if (local) {
      // (not produced by the API: phases carry no controls) a controlled
      // phase on a global target is a phase on the controls' set
      fail(QS_E_ARG, "controlled phase on a global qubit");
    }
    scalar = std::complex<double>(op.m[0], op.m[1]);
    return true;
  }
  if (pt >= m) fail(QS_E_ARG, "partition schedule: moved qubit is not local");
  out.t = pt;
  has_op = true;
  return true;
}

}  // namespace qs

using namespace qs;

extern "C" {

int partPlanSchedule(int numQubits, int globalQubits, const QSOp* ops, int64_t numOps, QSPartStep* steps,
                     int64_t maxSteps, int64_t* numSteps, int* finalPerm) {
  return guarded_call([&] {
    if (!numSteps || (numOps > 0 && !ops) || (maxSteps > 0 && !steps)) fail(QS_E_ARG, "null pointer");
    if (numQubits < 2 || numQubits > 40) fail(QS_E_QUBIT, "numQubits must be in 2..40");
    if (globalQubits < 1 || globalQubits >= numQubits) fail(QS_E_QUBIT, "globalQubits must be in 1..numQubits-1");
    Reg shape;
    shape.n = numQubits;
    shape.nq = numQubits;
    shape.prec = QS_C128;
    shape.dim = int64_t(1) << numQubits;
    std::vector<GateOp> g;
    convert_ops(shape, ops, numOps, g);
    std::vector<int> perm(static_cast<size_t>(numQubits));
    for (int q = 0; q < numQubits; ++q) perm[size_t(q)] = q;
    const std::vector<PartStep> st = plan_partition(numQubits, numQubits - globalQubits, g, perm);
    // LOCAL steps name the caller's op (one QSOp converts to one internal op)
    if (int64_t(g.size()) != numOps) fail(QS_E_ARG, "ops that expand to several gates");
    *numSteps = int64_t(st.size());
    if (int64_t(st.size()) > maxSteps && maxSteps > 0) fail(QS_E_ARG, "steps buffer too small");
    for (size_t i = 0; i < st.size() && int64_t(i) < maxSteps; ++i)
      steps[i] = QSPartStep{int32_t(st[i].kind), st[i].op, st[i].global_pos, st[i].local_pos};
    if (finalPerm)
      for (int q = 0; q < numQubits; ++q) finalPerm[q] = perm[size_t(q)];
  });
}

}  // extern "C"
