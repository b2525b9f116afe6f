// Flush of a register's queued gates.
#include "runtime.h"

namespace qs {

void flush(Reg& r) {
  if (r.queue.empty()) return;
  std::vector<GateOp> ops;
  ops.swap(r.queue);
  for (const GateOp& op : ops) launch_op(*r.env, r, op);
}

}  // namespace qs
