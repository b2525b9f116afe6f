// Host-side runtime structures of the simulator library (environment,
// registers, validated operations).  Internal: not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <functional>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "qsim.h"

namespace qs {

// A validated operation in the library's internal form.
enum class OpK : int32_t {
  GEN = 0,   // general 2x2 on t (m = re/im row-major: re0 im0 re1 im1 ...)
  H = 1,
  SX = 2,
  SY = 3,
  X = 4,
  PHASE = 5,    // diag(1, e^{i phi}) on t: m[0] = cos phi, m[1] = sin phi
  SIGN = 6,     // negate where every bit of cmask is set (t unused)
  DEPHASE = 7,  // density matrix only, p in m[0]
  DEPOL = 8,    // density matrix only, p in m[0]
  MULTI = 9     // dense 2^nt x 2^nt matrix on targets tg[0..nt) (matrix in big)
};

struct GateOp {
  OpK k;
  int t;            // target qubit (logical), -1 for SIGN
  uint64_t cmask;   // control bits (logical qubits); SIGN: the flipped set
  double m[8];
  int nt = 0;       // MULTI: number of targets
  uint8_t tg[8] = {};
  std::shared_ptr<const std::vector<double>> big;  // MULTI: row-major (re, im) matrix
};

struct Error {
  int code;
  std::string msg;
};
[[noreturn]] inline void fail(int code, const std::string& msg) { throw Error{code, msg}; }

#define QS_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      ::qs::fail(QS_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

struct Env;

// Per-kernel-class event timing (option "profile").
struct KStat {
  std::string name;
  int64_t launches = 0;
  double ms = 0, bytes = 0, flops = 0, alu = 0;
};
struct KPending {
  int cls;
  cudaEvent_t a, b;
};
struct Profiler {
  std::vector<KStat> stats;
  std::vector<KPending> pending;
  std::vector<cudaEvent_t> pool;
  int class_of(const std::string& name);
  cudaEvent_t event();
  void collect();  // caller has synchronised the stream
  void reset();
};

struct Reg {
  int64_t id = 0;
  Env* env = nullptr;
  int n = 0;          // logical qubits
  bool density = false;
  int nq = 0;         // qubits of the stored vector (n, or 2n for a density matrix)
  int prec = QS_C128;
  int64_t dim = 0;    // 2^nq amplitudes
  void* d = nullptr;  // amplitudes (double2 or float2)
  size_t bytes = 0;
  std::vector<GateOp> queue;  // gates waiting for a fused flush
  // Bits b of the stored index for which every amplitude with bit b set is
  // exactly 0: the register was zeroed and nothing since has mixed
  // amplitudes along b.  The planner turns gates on such bits into copies
  // or drops them.  Cleared whenever amplitudes are written from outside.
  uint64_t zero_bits = 0;
  // Scalar every amplitude is to be multiplied by: the factors that unfused
  // uncontrolled H / sqrt(X) / sqrt(Y) passes leave out (they apply the
  // matrices without them).  Applied at the next flush (by the fused plan's
  // final scale, or by one scaling pass), before anything reads the
  // amplitudes.
  std::complex<double> pend_scale{1.0, 0.0};
  // Per qubit t: a factor every amplitude with bit t set is to be multiplied
  // by (state vectors, unfused complex128 gates: the cos phi of a phase
  // applied as 1 + i tan phi, the output phase of a general update run as
  // phase-shear).  A real one is taken by the next uncontrolled H / sqrt(X)
  // / sqrt(Y) on t as its bit-1 input factor, any by the next uncontrolled
  // general update on t (folded into its matrix); applied before any other
  // update targeting t and at every flush.
  std::complex<double> qscale[64];
  Reg() {
    for (std::complex<double>& q : qscale) q = 1.0;
  }
  void reset_qscale() {
    for (std::complex<double>& q : qscale) q = 1.0;
  }
};

struct Env {
  int64_t id = 0;
  int device = 0;
  int sms = 148;
  cudaStream_t own = nullptr;
  cudaStream_t stream = nullptr;
  // options
  int64_t fusion = 1;
  int64_t tile_qubits = 0;
  int64_t max_fused_ops = 0;
  int64_t budget = 0;
  int64_t used = 0;
  int64_t profile = 0;
  int64_t arith = 0;         // complex128 arithmetic of fused passes: 0 = IEEE FP64, 1 = double-float
  int64_t multi_tc = 1;      // complex64 dense gates on 4-5 targets: 0 CUDA cores, 1 by shape (5 on the tensor cores), 2 tensor cores
  // batches built from now on: 0 = one launch per wave (graph of waves),
  // 1 = one persistent launch over every wave (k_fused_batch_persist; 69.0
  // against 73.1 ms for the 4096-register workload)
  int64_t batch_persistent = 1;
  // fused tiles: the lowest qubits every tile holds, i.e. the contiguous
  // HBM chunk of 2^L amplitudes (0 = 4 for complex64, 3 for complex128)
  int64_t tile_low_qubits = 0;
  // diagnostic of the persistent form's bounded wait: batches built while it
  // is 1 wait for one tile more than every previous pass has, with a 2 ms
  // bound, so every such wait runs out (QS_E_TIMEOUT at getBatchNorms)
  int64_t batch_diag_stall = 0;
  int64_t fused_cluster = 8;   // single-tile fused passes: largest thread-block cluster (CTAs, 2/4/8) they spread over, 0 or 1 = one CTA
  int64_t multi_tc_stage = 1;  // tensor-core multi-target passes with >= 7 free qubits: 1 staged (cp.async tiles, A in tensor memory), 0 register gather
  // fused passes as runtime-compiled kernels (jit.cpp): 0 off, 1 compile and
  // wait, 2 compile in the background (interpreting kernel until ready);
  // registers of at least jit_min_qubits stored qubits; CTAs per SM
  int64_t jit = 2;
  int64_t jit_min_qubits = 20;
  int64_t jit_ctas = 0;  // 0 = by shape (see jit_shape_for)
  // how generated kernels move tiles: 0 coalesced loads / stores, 1 bulk
  // (TMA) copies double-buffered, 2 asynchronous copies double-buffered,
  // -1 = by arithmetic (2 for complex64, 0 otherwise)
  int64_t jit_copy = -1;
  // the last stage of a generated pass stores straight to HBM (measured,
  // 30-qubit workload: complex64 9743 -> 10155 gates/s, double-float 1601
  // -> 1697)
  int64_t jit_direct = 1;
  // generated kernels swizzle the tile in shared memory (bank conflicts of
  // stages whose register bits hold the low local positions)
  int64_t jit_swizzle = 1;
  // IEEE-FP64 passes are bound by the FP64 pipe, where the interpreting
  // kernel measured faster (30 qubits: 83.4 vs 88.3 ms a pass): they use
  // generated kernels only when this is 1
  int64_t jit_fp64 = 0;
  // reuse of plans for repeated gate lists (fused.cu): on by default
  int64_t plan_cache_on = 1;
  int64_t plan_cache_hits = 0;
  std::shared_ptr<void> plan_cache;
  Profiler prof;
  // counters (readable through getEnvOption)
  int64_t launches = 0;      // kernel launches issued
  int64_t fused_passes = 0;  // fused-tile passes launched
  int64_t fused_vops = 0;    // vector operations applied by fused passes
  int64_t jit_launches = 0;  // fused passes launched as runtime-compiled kernels
  int64_t jit_rejected = 0;  // passes the kernel generator could not express
  // allocator hook
  void* (*alloc)(size_t, void*) = nullptr;
  void (*release)(void*, void*) = nullptr;
  void* actx = nullptr;
  // scratch: reduction partials and results (device), pinned result copy
  double* d_partial = nullptr;
  double* d_result = nullptr;
  double* h_result = nullptr;
  // device status word: kernels set bits when a bounded device wait runs
  // out; read (and cleared) at the next synchronisation, see check_status
  unsigned* d_status = nullptr;
  unsigned* h_status = nullptr;
  // staging buffer for complex64 <-> complex128 copies
  double2* d_stage = nullptr;
  int64_t stage_amps = 0;
  // fused-pass op and stage lists: pinned staging and device copies
  void* h_fops = nullptr;
  void* d_fops = nullptr;
  size_t fops_cap = 0;
  void* h_fst = nullptr;
  void* d_fst = nullptr;
  size_t fst_cap = 0;
  cudaEvent_t fcopied = nullptr;
  std::vector<int64_t> regs;
};

// Brackets one kernel launch with events when profiling is on: construct
// right before the launch, destroy right after it.  Counts launches always.
class KTimer {
 public:
  KTimer(Env& env, const char* name, double bytes, double flops, int nlaunch = 1, double alu = 0);
  ~KTimer();
  KTimer(const KTimer&) = delete;
  KTimer& operator=(const KTimer&) = delete;

 private:
  Env& env_;
  int cls_ = -1;
  cudaEvent_t a_ = nullptr;
};

// Fails with QS_E_TIMEOUT (and clears the word) if a kernel reported a
// bounded wait that ran out; h_status must have been copied from d_status
// and the stream synchronised.
void check_status(Env& env);
// Launches the bounded-wait diagnostic kernel (tc_multi.cuh).
void launch_wait_probe(Env& env, int timeout_us);

// Message returned by qsLastError on this thread (api.cu).
void set_last_error(const std::string& msg);
// Runs f, mapping exceptions to a status code and qsLastError (api.cu).
int guarded_call(const std::function<void()>& f);
// Handle lookups (api.cu); fail with QS_E_HANDLE when unknown.
Env& lookup_env(int64_t id);
Reg& lookup_reg(int64_t id);
// Queues (fusion on) or launches (fusion off) one validated op (api.cu).
void apply_op(Reg& r, const GateOp& op);
// Validation helpers (oplist.cpp): a qubit in [0, n) (QS_E_QUBIT); a
// target plus controls, in range and pairwise distinct (QS_E_DUP), as the
// control mask; a unitary 2x2 matrix, row-major (re, im) (QS_E_UNITARY).
void check_qubit(const Reg& r, int q, const char* what);
uint64_t check_targets(const Reg& r, int target, const int* ctrls, int nc);
void check_unitary(const double* m);
GateOp make_op(OpK k, int t, uint64_t cmask);
// Validates one bulk-call op, appending its internal ops (oplist.cpp).
void convert_op(const Reg& r, const QSOp& o, std::vector<GateOp>& out);
// Validates bulk-call ops for a register of r's shape into internal ops
// (oplist.cpp); fails with the first bad op's code.
void convert_ops(const Reg& r, const QSOp* ops, int64_t n, std::vector<GateOp>& out);

// Clears the bits of r.zero_bits that op mixes (planner.cpp): call after
// launching op outside a fused plan.
void note_mixing(Reg& r, const GateOp& op);

// Entry points of the kernel layer (implemented in the .cu files).
void launch_op(Env& env, Reg& r, const GateOp& op);
void flush(Reg& r);
void free_fused_buffers(Env& env);
double reduce_total(Env& env, Reg& r);
// Queue a reduction into the device double *out without waiting (serving).
void queue_total(Env& env, Reg& r, double* out);
void queue_outcome(Env& env, Reg& r, int q, int o, double* out);
double reduce_outcome(Env& env, Reg& r, int q, int o);
double reduce_purity(Env& env, Reg& r);
// <a|b> = sum_j conj(a_j) b_j in FP64 (state vectors of equal size, any
// precisions), on a's env stream; flushes both.
std::complex<double> reduce_inner(Env& env, Reg& a, Reg& b);
void launch_collapse(Env& env, Reg& r, int q, int o, double scale);
void launch_fill(Env& env, Reg& r, double re, double im);
// Multiplies every amplitude by f (settles Reg::pend_scale).
void launch_scale(Env& env, Reg& r, std::complex<double> f);
// Applies every pending Reg::qscale factor (launch.cu).
void settle_qscales(Reg& r);
void launch_convert(Env& env, const void* src, void* dst, int64_t count, bool to_double);

}  // namespace qs
