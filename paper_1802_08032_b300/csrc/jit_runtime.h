// Launch side of the runtime-compiled pass kernels (jit.cpp); internal.
#pragma once
#include <string>
#include <vector>

#include "plan.h"
#include "runtime.h"

namespace qs {

// Launches pass fp of register r with its generated kernel if the env's
// "jit" option allows it and the kernel is compiled (option 1 waits for the
// compile, option 2 queues it and returns false until it is ready).  st and
// ops are the plan's host arrays (fp's indices relative to them).  Returns
// false when the caller must launch the interpreting kernel instead.
bool jit_try_launch(Env& env, Reg& r, const FPass& fp, const FStage* st, const FOp* ops, Arith arith, int R,
                    double flops, double alu, const char* name);

// NVRTC compile of a generated source to an sm_103a cubin (no GPU needed).
bool jit_compile_cubin(const std::string& src, std::vector<char>& cubin, std::string& log);

struct JitStats {
  int64_t ready, pending, failed;
  double compile_s;  // summed compile + load time of the ready kernels
};
JitStats jit_stats();
std::string jit_first_failure();

}  // namespace qs
