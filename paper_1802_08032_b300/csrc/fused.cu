// Flush of a register's queued gates: fused-tile launches of the planned
// passes (the planner is in planner.cpp).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <memory>
#include <string>
#include <type_traits>
#include <unordered_map>

#include "fused_kernel.cuh"
#include "jit_runtime.h"
#include "plan.h"
#include "runtime.h"

namespace qs {

namespace {

// A single-tile pass on a cluster of C CTAs (k_fused_cluster).
template <class A, int R, int C>
void launch_cluster(Env& env, Reg& r, const FPass& fp, const FOp* d_ops, const FStage* d_st) {
  constexpr int c = C == 2 ? 1 : C == 4 ? 2 : 3;
  const size_t smem = cluster_smem_bytes<A>(fp.k, c, fp.L, fp.op_count, fp.stage_end - fp.stage_begin);
  static const bool attr_set = [] {
    QS_CUDA(cudaFuncSetAttribute(k_fused_cluster<A, R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 110 * 1024));
    return true;
  }();
  (void)attr_set;
  k_fused_cluster<A, R, C><<<C, (1 << (fp.k - R)) / C, smem, env.stream>>>(static_cast<typename A::Store*>(r.d), fp,
                                                                          d_ops, d_st);
}

template <class A, int R>
void launch_cluster_r(Env& env, Reg& r, const FPass& fp, const FOp* d_ops, const FStage* d_st, int ctas) {
  if (ctas == 8) launch_cluster<A, R, 8>(env, r, fp, d_ops, d_st);
  else if (ctas == 4) launch_cluster<A, R, 4>(env, r, fp, d_ops, d_st);
  else launch_cluster<A, R, 2>(env, r, fp, d_ops, d_st);
}

// A pass of a cluster plan (RegPlan::cluster > 1; plain arithmetic, R of
// the plan).
void launch_cluster_pass(Env& env, Reg& r, const RegPlan& pl, const FPass& fp, const FOp* d_ops,
                         const FStage* d_st, double flops, double alu, const char* name) {
  const double bytes = std::ldexp(2.0 * (pl.arith == Arith::F32 ? 8 : 16), r.nq);
  KTimer kt(env, name, bytes, flops, 1, alu);
  if (pl.arith == Arith::F64) {
    switch (pl.R) {
      case 2: return launch_cluster_r<PlainArith<double>, 2>(env, r, fp, d_ops, d_st, pl.cluster);
      case 3: return launch_cluster_r<PlainArith<double>, 3>(env, r, fp, d_ops, d_st, pl.cluster);
      case 4: return launch_cluster_r<PlainArith<double>, 4>(env, r, fp, d_ops, d_st, pl.cluster);
      default: break;
    }
  } else if (pl.arith == Arith::F32) {
    switch (pl.R) {
      case 2: return launch_cluster_r<PlainArith<float>, 2>(env, r, fp, d_ops, d_st, pl.cluster);
      case 3: return launch_cluster_r<PlainArith<float>, 3>(env, r, fp, d_ops, d_st, pl.cluster);
      case 4: return launch_cluster_r<PlainArith<float>, 4>(env, r, fp, d_ops, d_st, pl.cluster);
      case 5: return launch_cluster_r<PlainArith<float>, 5>(env, r, fp, d_ops, d_st, pl.cluster);
      default: break;
    }
  }
  fail(QS_E_ARG, "cluster plan with an unsupported arithmetic or register-bit count");
}

template <class A, int R>
void launch_pass(Env& env, Reg& r, const FPass& fp, const FOp* d_ops, const FStage* d_st,
                 double flops, double alu, const char* name) {
  const size_t smem = fused_smem_bytes<A>(fp.k, fp.L, fp.op_count, fp.stage_end - fp.stage_begin);
  // once per instantiation (thread-safe static initialisation)
  static const bool attr_set = [] {
    QS_CUDA(cudaFuncSetAttribute(k_fused<A, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 110 * 1024));
    return true;
  }();
  (void)attr_set;
  const int threads = 1 << (fp.k - R);
  const int64_t grid = std::min<int64_t>(fp.ntiles, int64_t(env.sms) * fused_ctas_per_sm(R));
  const double bytes = std::ldexp(2.0 * sizeof(typename A::Store), r.nq);
  KTimer kt(env, name, bytes, flops, 1, alu);
  k_fused<A, R><<<int(grid), threads, smem, env.stream>>>(static_cast<typename A::Store*>(r.d), fp,
                                                          d_ops, d_st);
}

// Grows the env's op / stage staging (pinned host + device) to fit.
void ensure_fused_buffers(Env& env, size_t nops, size_t nst) {
  if (env.fcopied) QS_CUDA(cudaEventSynchronize(env.fcopied));  // staging free to overwrite
  if (nops * sizeof(FOp) > env.fops_cap) {
    if (env.d_fops) { cudaFree(env.d_fops); cudaFreeHost(env.h_fops); env.d_fops = env.h_fops = nullptr; }
    env.fops_cap = std::max(nops, size_t(4096)) * sizeof(FOp);
    QS_CUDA(cudaMalloc(&env.d_fops, env.fops_cap));
    QS_CUDA(cudaMallocHost(&env.h_fops, env.fops_cap));
  }
  if (nst * sizeof(FStage) > env.fst_cap) {
    if (env.d_fst) { cudaFree(env.d_fst); cudaFreeHost(env.h_fst); env.d_fst = env.h_fst = nullptr; }
    env.fst_cap = std::max(nst, size_t(1024)) * sizeof(FStage);
    QS_CUDA(cudaMalloc(&env.d_fst, env.fst_cap));
    QS_CUDA(cudaMallocHost(&env.h_fst, env.fst_cap));
  }
  if (!env.fcopied) QS_CUDA(cudaEventCreateWithFlags(&env.fcopied, cudaEventDisableTiming));
}

// Plans of recently flushed gate lists.  A plan is a pure function of the
// gate list and of what build_plan reads besides (register shape and
// precision, arithmetic, tile-size and depth options, known-zero bits,
// pending scalar), so a repeated flush of the same list reuses it instead of
// re-planning (the 30-qubit workload plans in ~0.6 ms, the 12-qubit one in
// ~40 us of a ~260 us circuit).
struct PlanCacheImpl {
  struct Entry {
    RegPlan plan;
    uint64_t used = 0;
  };
  std::unordered_map<std::string, Entry> map;
  uint64_t tick = 0;
  static constexpr size_t kEntries = 16;
};

template <typename T>
void put(std::string& k, const T& v) {
  k.append(reinterpret_cast<const char*>(&v), sizeof(T));
}

std::string plan_key(const Reg& r, const std::vector<GateOp>& seg, int k_req, uint64_t zero_in,
                     std::complex<double> scale) {
  const Env& env = *r.env;
  std::string k;
  k.reserve(64 + seg.size() * 96);
  put(k, k_req);
  put(k, r.nq);
  put(k, r.n);
  put(k, r.density);
  put(k, r.prec);
  put(k, int(arith_of(r)));
  put(k, env.tile_qubits);
  put(k, env.max_fused_ops);
  put(k, env.fused_cluster);
  put(k, env.tile_low_qubits);
  put(k, zero_in);
  put(k, scale.real());
  put(k, scale.imag());
  for (const GateOp& op : seg) {
    put(k, op.k);
    put(k, op.t);
    put(k, op.cmask);
    k.append(reinterpret_cast<const char*>(op.m), sizeof(op.m));
  }
  return k;
}

// build_plan through the env's plan cache.  Passes that will run as
// generated kernels with a copy pipeline get tiles that leave room for two
// buffers (unless the env fixes the tile size).
void cached_plan(Reg& r, const std::vector<GateOp>& seg, uint64_t zero_in, std::complex<double> scale,
                 RegPlan& out) {
  Env& env = *r.env;
  const int k_req = env.tile_qubits > 0 ? 0 : jit_tile_cap(env, r, arith_of(r));
  if (!env.plan_cache_on) {
    build_plan(r, seg, k_req, zero_in, scale, out);
    return;
  }
  if (!env.plan_cache) env.plan_cache = std::make_shared<PlanCacheImpl>();
  PlanCacheImpl& c = *static_cast<PlanCacheImpl*>(env.plan_cache.get());
  std::string key = plan_key(r, seg, k_req, zero_in, scale);
  auto it = c.map.find(key);
  if (it != c.map.end()) {
    it->second.used = ++c.tick;
    out = it->second.plan;
    for (FPass& fp : out.fps) fp.amps = r.d;
    ++env.plan_cache_hits;
    return;
  }
  build_plan(r, seg, k_req, zero_in, scale, out);
  if (c.map.size() >= PlanCacheImpl::kEntries) {
    auto lru = c.map.begin();
    for (auto e = c.map.begin(); e != c.map.end(); ++e)
      if (e->second.used < lru->second.used) lru = e;
    c.map.erase(lru);
  }
  PlanCacheImpl::Entry& e = c.map[std::move(key)];
  e.plan = out;
  e.used = ++c.tick;
}

}  // namespace

void free_fused_buffers(Env& env) {
  if (env.fcopied) cudaEventSynchronize(env.fcopied);
  if (env.d_fops) { cudaFree(env.d_fops); cudaFreeHost(env.h_fops); }
  if (env.d_fst) { cudaFree(env.d_fst); cudaFreeHost(env.h_fst); }
  if (env.fcopied) cudaEventDestroy(env.fcopied);
  env.d_fops = env.h_fops = env.d_fst = env.h_fst = nullptr;
  env.fops_cap = env.fst_cap = 0;
  env.fcopied = nullptr;
}

// Applies a pending scalar factor the fused plans did not absorb.
void settle_scale(Reg& r) {
  if (r.pend_scale == std::complex<double>(1.0, 0.0)) return;
  launch_scale(*r.env, r, r.pend_scale);
  r.pend_scale = 1.0;
}

void flush(Reg& r) {
  // deferred per-qubit factors of unfused phases first (the plans assume none)
  if (!r.density) settle_qscales(r);
  if (r.queue.empty()) {
    settle_scale(r);
    return;
  }
  std::vector<GateOp> q;
  q.swap(r.queue);
  Env& env = *r.env;
  if (!fusable(r)) {
    for (const GateOp& op : q) {
      launch_op(env, r, op);
      note_mixing(r, op);
    }
    if (!r.density) settle_qscales(r);
    settle_scale(r);
    return;
  }
  // Multi-target gates run as their own passes; the gates between them form
  // fused segments.  All segments' op lists go up in one copy.
  std::vector<RegPlan> plans;
  std::vector<int> after;  // index into q of the multi-target gate following each plan, or -1
  std::vector<GateOp> seg;
  // the known-zero bits flow through the plans and the multi-target gates
  auto close = [&](int next) {
    if (!seg.empty()) {
      plans.emplace_back();
      // the pending factor rides on the first plan's final scale (all ops are linear)
      cached_plan(r, seg, r.zero_bits, r.pend_scale, plans.back());
      r.zero_bits = plans.back().zero_out;
      if (!plans.back().fps.empty()) r.pend_scale = 1.0;
      after.push_back(next);
      seg.clear();
    } else if (next >= 0) {
      plans.emplace_back();  // empty plan: only the multi-target gate
      after.push_back(next);
    }
    if (next >= 0) note_mixing(r, q[size_t(next)]);
  };
  for (size_t i = 0; i < q.size(); ++i) {
    if (q[i].k == OpK::MULTI) close(int(i));
    else seg.push_back(q[i]);
  }
  close(-1);
  size_t nops = 0, nst = 0;
  for (const RegPlan& pl : plans) {
    nops += pl.fops.size();
    nst += pl.fst.size();
  }
  std::vector<size_t> op0, st0;
  if (nops > 0) {
    ensure_fused_buffers(env, nops, nst);
    FOp* hops = static_cast<FOp*>(env.h_fops);
    FStage* hst = static_cast<FStage*>(env.h_fst);
    size_t o = 0, s = 0;
    for (const RegPlan& pl : plans) {
      op0.push_back(o);
      st0.push_back(s);
      std::memcpy(hops + o, pl.fops.data(), pl.fops.size() * sizeof(FOp));
      std::memcpy(hst + s, pl.fst.data(), pl.fst.size() * sizeof(FStage));
      o += pl.fops.size();
      s += pl.fst.size();
    }
    QS_CUDA(cudaMemcpyAsync(env.d_fops, env.h_fops, nops * sizeof(FOp), cudaMemcpyHostToDevice, env.stream));
    QS_CUDA(cudaMemcpyAsync(env.d_fst, env.h_fst, nst * sizeof(FStage), cudaMemcpyHostToDevice, env.stream));
    QS_CUDA(cudaEventRecord(env.fcopied, env.stream));
  }
  for (size_t pi = 0; pi < plans.size(); ++pi) {
    const RegPlan& pl = plans[pi];
    env.fused_passes += int64_t(pl.fps.size());
    env.fused_vops += pl.vops;
    for (size_t i = 0; i < pl.fps.size(); ++i) {
      FPass fp = pl.fps[i];
      fp.op_begin += int(op0[pi]);
      fp.stage_begin += int(st0[pi]);
      fp.stage_end += int(st0[pi]);
      const FOp* d_ops = static_cast<const FOp*>(env.d_fops);
      const FStage* d_st = static_cast<const FStage*>(env.d_fst);
      const char* name = pl.arith == Arith::DF ? "fused_c128_df" : pl.arith == Arith::F64 ? "fused_c128" : "fused_c64";
      if (pl.cluster > 1) {  // one tile on a thread-block cluster
        launch_cluster_pass(env, r, pl, fp, d_ops, d_st, pl.flops[i], pl.alu[i], name);
        continue;
      }
      // the pass as its own compiled kernel when one is ready (jit.cpp)
      const int R = pl.arith == Arith::F32 ? 5 : 4;
      if (jit_try_launch(env, r, pl.fps[i], pl.fst.data(), pl.fops.data(), pl.arith, R, pl.flops[i], pl.alu[i], name,
                         pl.jit_memo.get(), i))
        continue;
      if (pl.arith == Arith::DF)
        launch_pass<DFArith, 4>(env, r, fp, d_ops, d_st, pl.flops[i], pl.alu[i], "fused_c128_df");
      else if (pl.arith == Arith::F64)
        launch_pass<PlainArith<double>, 4>(env, r, fp, d_ops, d_st, pl.flops[i], pl.alu[i], "fused_c128");
      else
        launch_pass<PlainArith<float>, 5>(env, r, fp, d_ops, d_st, pl.flops[i], pl.alu[i], "fused_c64");
    }
    if (after[pi] >= 0) {
      launch_op(env, r, q[size_t(after[pi])]);
      // (a one-target gate runs as a pair update and may leave a per-qubit
      // factor; the next plan and every read assume none)
      if (!r.density) settle_qscales(r);
    }
  }
  settle_scale(r);
  QS_CUDA(cudaGetLastError());
}

}  // namespace qs
