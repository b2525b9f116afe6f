// Pass kernels compiled at run time for one fused pass's operation list.
//
// The fused tile kernel (fused_kernel.cuh) interprets a pass: every thread
// decodes every operation (dispatch word, condition masks, pending sign
// flips) before its arithmetic, which for complex64 costs more instructions
// than the arithmetic itself.  A pass's structure (tile qubits, stages,
// operation kinds, register bits, condition masks) is fixed once planned, so
// this module writes a kernel with that structure spelled out in straight-
// line code, compiles it with NVRTC for sm_103a and caches it by its source
// text.  Coefficients stay kernel parameters (the pass's FOp array, read from
// the constant bank), so a circuit rerun with other angles reuses the
// kernels.  The arithmetic is the same inline code as the interpreter's
// (fused_arith.cuh), applied in the same order; sign flips, which commute
// exactly with what they are moved past, are applied where they occur.
#pragma once
#include <cstdint>
#include <string>

#include "fused_types.h"
#include "plan.h"

namespace qs {

enum class JitCopy { Plain = 0, Bulk = 1, Async = 2 };

// Parameters of one generated pass kernel.
struct JitShape {
  Arith arith;
  int R;
  int ctas;  // resident CTAs per SM the kernel is compiled for (__launch_bounds__)
  // How tiles move between global and shared memory: Plain = coalesced
  // loads and stores through registers; Bulk = bulk (TMA) copies of the
  // tile's contiguous chunks through two shared-memory buffers, the next
  // tile's load overlapping the current tile's work (the kernel then takes a
  // device status word after ntiles: bit 1 = a copy did not arrive within 1 s
  // of the GPU's global timer); Async = the same double buffering with
  // 16-byte asynchronous copies (cp.async) in the plain access pattern.
  JitCopy copy = JitCopy::Plain;
  // the last stage of a pass writes its register amplitudes straight to
  // HBM instead of through shared memory (not with JitCopy::Bulk)
  bool direct_store = false;
  // the tile's shared-memory layout is XOR-swizzled against bank conflicts
  // (not with JitCopy::Bulk, whose chunks are copied whole)
  bool swizzle = false;
};

// CUDA source of the pass kernel `qs_pass` for pass fp of a plan whose
// stage and op arrays are st and ops (fp's indices relative to them).
// Kernel signature: (Store* g, long long ntiles, [unsigned* status,] const
// __grid_constant__ JitOps P) with P holding fp.op_count FOp records (the
// status word only with JitCopy::Bulk).  Throws Error (QS_E_ARG) if the pass uses a
// form the generator does not know.
std::string jit_source(const FPass& fp, const FStage* st, const FOp* ops, const JitShape& sh);

// Shared-memory bytes of a generated pass kernel.
size_t jit_smem_bytes(const FPass& fp, const JitShape& sh);

// Headers the generated source includes, as (name, contents) pairs embedded
// at build time; used by the NVRTC compile.
int jit_header_count();
const char* jit_header_name(int i);
const char* jit_header_text(int i);

}  // namespace qs
