// Partitioned state vectors (the paper's distributed scheme, Sec. II.B.2):
// internal declarations shared by the schedule planner (partition.cpp, host
// only) and the executor (partition.cu).
//
// An n-qubit state vector is held as P = 2^k parts of 2^m amplitudes
// (m = n - k local qubits): physical index bits below m address a part's
// amplitudes, bits m..n-1 name the part.  Gates that move amplitudes
// along a qubit (every non-diagonal update) need that qubit at a local
// position; a gate on a global one is preceded by a qubit swap that brings
// it to a local position (each part exchanges half of its amplitudes with
// the part that differs in that global bit), after which the gate and the
// fused tiles that follow run inside each part.  Diagonal gates and
// controls on global qubits need no exchange: a part knows its global bits,
// so they become per-part predicates or scalars.
#pragma once
#include <cstdint>
#include <vector>

#include "runtime.h"

namespace qs {

// One step of a partitioned circuit.
struct PartStep {
  enum Kind : int32_t { LOCAL = 0, SWAP = 1 } kind;
  int32_t op;         // LOCAL: index of the gate in the circuit
  int32_t global_pos; // SWAP: physical global position (m..n-1)
  int32_t local_pos;  // SWAP: physical local position (0..m-1)
};

// Plans a circuit on n logical qubits over parts of m local qubits, from the
// logical -> physical map perm (updated in place to the map after the
// circuit).  A swap brings each global target into the local position whose
// qubit is next moved furthest in the future (never = best).  Fails with
// QS_E_ARG for multi-target gates or channels.
std::vector<PartStep> plan_partition(int n, int m, const std::vector<GateOp>& ops, std::vector<int>& perm);

// The gate a part applies for logical gate op under map perm, or false when
// the part skips it (a control on a global qubit whose bit is 0 for this
// part); a gate whose qubits are all global and satisfied becomes a scalar
// factor (*scalar, with *has_op false).
bool part_gate(const GateOp& op, const std::vector<int>& perm, int m, int64_t part, GateOp& out, bool& has_op,
               std::complex<double>& scalar);

}  // namespace qs
