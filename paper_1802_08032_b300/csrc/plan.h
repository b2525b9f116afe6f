// Fusion plan of one register's queued gates (internal; planner.cpp).
#pragma once
#include <memory>
#include <vector>

#include "fused_types.h"
#include "runtime.h"

namespace qs {

// Coefficient form of the kernel's arithmetic.
enum class Arith { F32, F64, DF };

// The passes of one register: device-ready descriptors whose op and stage
// indices are relative to this plan's own arrays.
struct RegPlan {
  int k = 0, L = 0, R = 0;
  // > 1: the register is one tile, spread over a thread-block cluster of
  // this many CTAs (k_fused_cluster), with R chosen for 4 warps a CTA
  int cluster = 0;
  Arith arith = Arith::F64;
  std::vector<FPass> fps;
  std::vector<FOp> fops;
  std::vector<FStage> fst;
  std::vector<double> flops;  // algorithmic flops per pass
  std::vector<double> alu;    // arithmetic instructions per pass (kernel precision)
  int64_t vops = 0;           // vector operations planned
  uint64_t zero_out = 0;      // bits known to hold only zeros after the plan
  // generated kernels found for this plan's passes (jit.cpp), shared by the
  // copies the plan cache hands out, so a repeated plan skips generating
  // and looking up their sources; valid for the kernel shape `sig`
  struct JitMemo {
    uint64_t sig = 0;
    std::vector<std::shared_ptr<void>> kernels;
  };
  std::shared_ptr<JitMemo> jit_memo = std::make_shared<JitMemo>();
};

// Tile parameters per precision: R register bits, maximum k, low qubits L.
struct TileCfg {
  int R, kmax, L;
};
TileCfg tile_cfg(const Reg& r);
bool fusable(const Reg& r);
Arith arith_of(const Reg& r);

// Plans q for register r with tile size k (0 = the library default / the
// env's tile_qubits option).
// zero_in: bits known to hold only zeros before q (see Reg::zero_bits); the
// bits still known zero after q are returned in out.zero_out.
// scale_in: a scalar to apply to the whole register as well (folded into
// the plan's final scale when the plan has passes).
void build_plan(const Reg& r, const std::vector<GateOp>& q, int k_req, uint64_t zero_in,
                std::complex<double> scale_in, RegPlan& out);

}  // namespace qs
