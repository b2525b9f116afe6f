// Launch side of the runtime-compiled pass kernels (jit.cpp); internal.
#pragma once
#include <string>
#include <vector>

#include "jit.h"
#include "plan.h"
#include "runtime.h"

namespace qs {

// Launches pass fp of register r with its generated kernel if the env's
// "jit" option allows it and the kernel is compiled (option 1 waits for the
// compile, option 2 queues it and returns false until it is ready).  st and
// ops are the plan's host arrays (fp's indices relative to them).  Returns
// false when the caller must launch the interpreting kernel instead.
bool jit_try_launch(Env& env, Reg& r, const FPass& fp, const FStage* st, const FOp* ops, Arith arith, int R,
                    double flops, double alu, const char* name, RegPlan::JitMemo* memo = nullptr,
                    size_t pass_index = 0);

// True when passes of register r are to run as generated kernels (the
// env's "jit" options), so that the planner can size tiles for them.
inline bool jit_wanted(const Env& env, const Reg& r, Arith arith) {
  return env.jit != 0 && r.nq >= env.jit_min_qubits && (arith != Arith::F64 || env.jit_fp64 != 0);
}

// How generated kernels move tiles: the option, else by arithmetic.
// Measured on the 30-qubit workload (gates/s): complex64 coalesced loads
// 8512, bulk copies 8059, async copies 9743 (tiles of 2^12, 3 CTAs per SM);
// double-float 1601 / 1315 / 1354 (its passes are FP32-issue bound).
inline JitCopy jit_copy_mode(const Env& env, Arith arith) {
  if (env.jit_copy >= 0) return static_cast<JitCopy>(env.jit_copy);
  return arith == Arith::F32 ? JitCopy::Async : JitCopy::Plain;
}

// Resident CTAs per SM of a generated kernel: the option, else what shared
// memory and registers allow (complex64 with two 32 KiB buffers: 3).
inline int jit_ctas_for(const Env& env, const FPass& fp, Arith arith, JitCopy copy) {
  if (env.jit_ctas > 0) return int(env.jit_ctas);
  if (copy != JitCopy::Plain && arith == Arith::F32 && fp.k <= 12) return 3;
  return 2;
}

// Tile size cap of plans whose passes may run as generated kernels:
// complex64 tiles of 2^12 amplitudes (32 KiB) with a copy pipeline, so that
// two buffers each for three CTAs fit an SM's shared memory; 0 = no cap.
// It does not depend on whether generated kernels are on, or compiled yet:
// a register's plan, and so its rounding, is the same either way (the
// interpreting and generated kernels then agree bit for bit).
inline int jit_tile_cap(const Env& env, const Reg& r, Arith arith) {
  if (r.nq < env.jit_min_qubits) return 0;
  return arith == Arith::F32 && jit_copy_mode(env, arith) != JitCopy::Plain ? 12 : 0;
}

// NVRTC compile of a generated source to an sm_103a cubin (no GPU needed).
bool jit_compile_cubin(const std::string& src, std::vector<char>& cubin, std::string& log);

struct JitStats {
  int64_t ready, pending, failed;
  double compile_s;  // summed compile + load time of the ready kernels
};
JitStats jit_stats();
// Stops the background compile threads after the compiles in flight (called
// when the last environment is destroyed, and by qsJitShutdown).
void jit_shutdown();
std::string jit_first_failure();

}  // namespace qs
