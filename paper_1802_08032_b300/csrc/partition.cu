// Partitioned state vectors: the executor (see partition.h for the scheme
// and partition.cpp for the schedule).
//
// The P = 2^k parts are ordinary registers of m = n - k qubits on the
// env's device and stream; in the paper's deployment each would live on
// its own node or GPU.  A qubit swap between global position g and local
// position l pairs part p (bit g - m of p clear) with part p' (set): p keeps
// its amplitudes with bit l = 0 and sends the half with bit l = 1, p'
// keeps bit l = 1 and sends bit l = 0; each packs the half it sends into a
// send buffer, the buffers are exchanged (here a device-to-device copy into
// the partner's receive buffer: the step a multi-GPU deployment carries out
// with a point-to-point transfer), and each unpacks what it received into
// the half it sent.  Everything is queued on the env's stream in order, so
// no kernel waits for another.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "partition.h"
#include "runtime.h"

namespace qs {

namespace {

constexpr int kPartThreads = 256;

// buf[i] = a[j] (PACK) or a[j] = buf[i] (unpack), j = i with bit l = v
// inserted: the half of a part whose bit l equals v, in index order.
template <typename R, bool PACK>
__global__ void __launch_bounds__(kPartThreads) k_half(cvec<R>* __restrict__ a, cvec<R>* __restrict__ buf,
                                                      int64_t nhalf, int l, int v) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int64_t low = (int64_t(1) << l) - 1;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nhalf; i += stride) {
    const int64_t j = ((i & ~low) << 1) | (int64_t(v) << l) | (i & low);
    if (PACK) buf[i] = a[j];
    else a[j] = buf[i];
  }
}

struct PartReg {
  int64_t id = 0;
  Env* env = nullptr;
  int n = 0, k = 0, m = 0, prec = QS_C128;
  std::vector<Qureg> parts;
  std::vector<int> perm;         // logical qubit -> physical position
  void* buf[4] = {};             // send / receive halves of the two parts of a pair
  int64_t swaps = 0;
  double exchanged = 0;          // bytes moved between parts by swaps
};

std::mutex g_pmu;
std::unordered_map<int64_t, PartReg*> g_parts;
int64_t g_next_part = 1;

PartReg& part_of(QSPartReg h) {
  std::lock_guard<std::mutex> lk(g_pmu);
  auto it = g_parts.find(h.id);
  if (it == g_parts.end()) fail(QS_E_HANDLE, "unknown partitioned register " + std::to_string(h.id));
  return *it->second;
}

template <typename R>
void half_copy(Env& env, void* part, void* buf, int64_t nhalf, int l, int v, bool pack) {
  const int grid = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(env.sms) * 8,
                                                              (nhalf + kPartThreads - 1) / kPartThreads)));
  KTimer kt(env, pack ? "part_pack" : "part_unpack", double(nhalf) * 2 * sizeof(cvec<R>), 0);
  if (pack)
    k_half<R, true><<<grid, kPartThreads, 0, env.stream>>>(static_cast<cvec<R>*>(part), static_cast<cvec<R>*>(buf),
                                                          nhalf, l, v);
  else
    k_half<R, false><<<grid, kPartThreads, 0, env.stream>>>(static_cast<cvec<R>*>(part),
                                                           static_cast<cvec<R>*>(buf), nhalf, l, v);
  QS_CUDA(cudaGetLastError());
}

// Swaps physical positions g (global) and l (local) across every pair.
void run_swap(PartReg& P, int g, int l) {
  Env& env = *P.env;
  const int64_t nhalf = int64_t(1) << (P.m - 1);
  const size_t S = P.prec == QS_C128 ? 16 : 8;
  const int64_t bit = int64_t(1) << (g - P.m);
  for (Qureg q : P.parts) flush(lookup_reg(q.id));
  for (int64_t p0 = 0; p0 < int64_t(P.parts.size()); ++p0) {
    if (p0 & bit) continue;
    Reg& a = lookup_reg(P.parts[size_t(p0)].id);
    Reg& b = lookup_reg(P.parts[size_t(p0 | bit)].id);
    const bool c128 = P.prec == QS_C128;
    // pack: a sends its bit-l = 1 half, b its bit-l = 0 half
    if (c128) {
      half_copy<double>(env, a.d, P.buf[0], nhalf, l, 1, true);
      half_copy<double>(env, b.d, P.buf[1], nhalf, l, 0, true);
    } else {
      half_copy<float>(env, a.d, P.buf[0], nhalf, l, 1, true);
      half_copy<float>(env, b.d, P.buf[1], nhalf, l, 0, true);
    }
    // exchange: each send buffer into the partner's receive buffer
    QS_CUDA(cudaMemcpyAsync(P.buf[3], P.buf[0], size_t(nhalf) * S, cudaMemcpyDeviceToDevice, env.stream));
    QS_CUDA(cudaMemcpyAsync(P.buf[2], P.buf[1], size_t(nhalf) * S, cudaMemcpyDeviceToDevice, env.stream));
    // unpack into the halves that were sent
    if (c128) {
      half_copy<double>(env, a.d, P.buf[2], nhalf, l, 1, false);
      half_copy<double>(env, b.d, P.buf[3], nhalf, l, 0, false);
    } else {
      half_copy<float>(env, a.d, P.buf[2], nhalf, l, 1, false);
      half_copy<float>(env, b.d, P.buf[3], nhalf, l, 0, false);
    }
    a.zero_bits = 0;  // amplitudes written from outside the planner's view
    b.zero_bits = 0;
    P.exchanged += 2.0 * double(nhalf) * double(S);
  }
  ++P.swaps;
}

void destroy_part(PartReg* P) {
  for (Qureg q : P->parts)
    if (q.id) destroyQureg(q);
  for (void*& b : P->buf)
    if (b) {
      cudaFree(b);
      b = nullptr;
    }
  delete P;
}

}  // namespace

}  // namespace qs

using namespace qs;

extern "C" {

int createPartitionedQureg(int numQubits, int globalQubits, int precision, QuESTEnv env, QSPartReg* out) {
  return guarded_call([&] {
    if (!out) fail(QS_E_ARG, "null output");
    if (precision != QS_C64 && precision != QS_C128) fail(QS_E_ARG, "precision must be QS_C64 or QS_C128");
    if (numQubits < 2 || numQubits > 40) fail(QS_E_QUBIT, "numQubits must be in 2..40");
    if (globalQubits < 1 || globalQubits > 6 || globalQubits >= numQubits)
      fail(QS_E_QUBIT, "globalQubits must be in 1..min(6, numQubits - 1)");
    Env& e = lookup_env(env.id);
    auto* P = new PartReg();
    P->env = &e;
    P->n = numQubits;
    P->k = globalQubits;
    P->m = numQubits - globalQubits;
    P->prec = precision;
    try {
      for (int q = 0; q < numQubits; ++q) P->perm.push_back(q);
      for (int p = 0; p < (1 << globalQubits); ++p) {
        Qureg q{0};
        const int st = createQureg(P->m, precision, env, &q);
        if (st != QS_OK) fail(st, qsLastError());
        P->parts.push_back(q);
        // |0...0> lives in part 0; every other part starts at zero
        if (p > 0) {
          Reg& r = lookup_reg(q.id);
          QS_CUDA(cudaMemsetAsync(r.d, 0, r.bytes, e.stream));
          r.zero_bits = 0;
        }
      }
      const size_t half = (size_t(1) << (P->m - 1)) * (precision == QS_C128 ? 16 : 8);
      for (void*& b : P->buf) QS_CUDA(cudaMalloc(&b, half));
    } catch (...) {
      destroy_part(P);
      throw;
    }
    std::lock_guard<std::mutex> lk(g_pmu);
    P->id = g_next_part++;
    g_parts[P->id] = P;
    out->id = P->id;
  });
}

int destroyPartitionedQureg(QSPartReg h) {
  return guarded_call([&] {
    PartReg& P = part_of(h);
    cudaStreamSynchronize(P.env->stream);
    {
      std::lock_guard<std::mutex> lk(g_pmu);
      g_parts.erase(P.id);
    }
    destroy_part(&P);
  });
}

int partApplyCircuit(QSPartReg h, const QSOp* ops, int64_t numOps) {
  return guarded_call([&] {
    PartReg& P = part_of(h);
    if (numOps < 0 || (numOps > 0 && !ops)) fail(QS_E_ARG, "bad op list");
    Reg shape;
    shape.n = P.n;
    shape.nq = P.n;
    shape.prec = P.prec;
    shape.dim = int64_t(1) << P.n;
    std::vector<GateOp> g;
    convert_ops(shape, ops, numOps, g);
    std::vector<int> perm = P.perm;
    const std::vector<PartStep> steps = plan_partition(P.n, P.m, g, perm);
    for (const PartStep& s : steps) {
      if (s.kind == PartStep::SWAP) {
        run_swap(P, s.global_pos, s.local_pos);
        // the map moves with the swap: the two positions trade qubits
        for (int& x : P.perm) {
          if (x == s.global_pos) x = s.local_pos;
          else if (x == s.local_pos) x = s.global_pos;
        }
        continue;
      }
      const GateOp& op = g[size_t(s.op)];
      for (int64_t p = 0; p < int64_t(P.parts.size()); ++p) {
        GateOp lop;
        bool has_op = false;
        std::complex<double> scalar;
        if (!part_gate(op, P.perm, P.m, p, lop, has_op, scalar)) continue;
        Reg& r = lookup_reg(P.parts[size_t(p)].id);
        if (has_op) apply_op(r, lop);
        else r.pend_scale *= scalar;  // applied by the part's next flush
      }
    }
    if (P.perm != perm) fail(QS_E_ARG, "partition map out of step with its schedule");
  });
}

int partCalcTotalProb(QSPartReg h, double* out) {
  return guarded_call([&] {
    if (!out) fail(QS_E_ARG, "null output");
    PartReg& P = part_of(h);
    // each part reduces in FP64; the parts' sums add in part order (the
    // all-reduce of a distributed run)
    double s = 0;
    for (Qureg q : P.parts) {
      double t = 0;
      const int st = calcTotalProb(q, &t);
      if (st != QS_OK) fail(st, qsLastError());
      s += t;
    }
    *out = s;
  });
}

int partCalcProbOfOutcome(QSPartReg h, int qubit, int outcome, double* out) {
  return guarded_call([&] {
    if (!out) fail(QS_E_ARG, "null output");
    PartReg& P = part_of(h);
    if (qubit < 0 || qubit >= P.n) fail(QS_E_QUBIT, "qubit out of range");
    if (outcome != 0 && outcome != 1) fail(QS_E_PROB, "outcome must be 0 or 1");
    const int pos = P.perm[size_t(qubit)];
    double s = 0;
    for (int64_t p = 0; p < int64_t(P.parts.size()); ++p) {
      double t = 0;
      int st;
      if (pos < P.m) {
        st = calcProbOfOutcome(P.parts[size_t(p)], pos, outcome, &t);
      } else {
        if (((p >> (pos - P.m)) & 1) != outcome) continue;
        st = calcTotalProb(P.parts[size_t(p)], &t);
      }
      if (st != QS_OK) fail(st, qsLastError());
      s += t;
    }
    *out = s;
  });
}

int partCopyStateToHost(QSPartReg h, Complex* dst) {
  return guarded_call([&] {
    if (!dst) fail(QS_E_ARG, "null output");
    PartReg& P = part_of(h);
    const int64_t np = int64_t(1) << P.m;
    std::vector<Complex> part(static_cast<size_t>(np));
    for (int64_t p = 0; p < int64_t(P.parts.size()); ++p) {
      const int st = copyStateToHost(P.parts[size_t(p)], part.data(), 0, np);
      if (st != QS_OK) fail(st, qsLastError());
      // physical index (p, j) -> logical index: bit perm[q] of the physical
      // index is bit q of the logical one
      const int64_t phys_hi = p << P.m;
      for (int64_t j = 0; j < np; ++j) {
        const int64_t phys = phys_hi | j;
        int64_t logical = 0;
        for (int q = 0; q < P.n; ++q) logical |= ((phys >> P.perm[size_t(q)]) & 1) << q;
        dst[logical] = part[size_t(j)];
      }
    }
  });
}

int partGetInfo(QSPartReg h, int* numQubits, int* globalQubits, int* perm, int64_t* swaps, double* exchangedBytes) {
  return guarded_call([&] {
    PartReg& P = part_of(h);
    if (numQubits) *numQubits = P.n;
    if (globalQubits) *globalQubits = P.k;
    if (perm)
      for (int q = 0; q < P.n; ++q) perm[q] = P.perm[size_t(q)];
    if (swaps) *swaps = P.swaps;
    if (exchangedBytes) *exchangedBytes = P.exchanged;
  });
}

}  // extern "C"
