// Batched engine: many independent registers advanced together.
//
// createBatch takes registers with queued gates (typically thousands of
// small state vectors of different sizes), plans each register's fused
// passes exactly as a single-register flush would, and lays the work out in
// waves: wave w holds pass w of every register that has one, as a list of
// (pass, tile) items.  One launch of k_fused_batch per wave runs every item
// of the wave; registers of up to 2^k amplitudes are a single tile, so they
// stay in shared memory for a whole pass, and the first pass generates
// |0...0> instead of reading memory.  The launches (plus one FP64 norm per
// register) are captured once into a CUDA graph; runBatch replays it.
// Waves follow one another in stream order, so no kernel ever waits on
// another kernel's progress.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "fused_kernel.cuh"
#include "plan.h"
#include "runtime.h"

namespace qs {

namespace {

constexpr int kNormThreads = 256;

struct NormDesc {
  const void* amps;
  int64_t dim;
};

__device__ __forceinline__ double norm_block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

// out[r] = sum |a_j|^2 of register r (one CTA per register, fixed order).
template <typename V>
__global__ void __launch_bounds__(kNormThreads) k_batch_norms(const NormDesc* __restrict__ regs,
                                                              double* __restrict__ out) {
  __shared__ double sh[32];
  const NormDesc d = regs[blockIdx.x];
  const V* a = static_cast<const V*>(d.amps);
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < d.dim; j += kNormThreads) {
    const V v = a[j];
    const double re = widen(v.x), im = widen(v.y);
    acc = fma(re, re, acc);
    acc = fma(im, im, acc);
  }
  const double s = norm_block_sum(acc, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

struct Wave {
  int first_item = 0, nitems = 0;
  int kmax = 0, Lmin = 64, opmax = 0, stmax = 0;
  double bytes = 0, flops = 0, alu = 0;
};

struct Batch {
  int64_t id = 0;
  Env* env = nullptr;
  std::vector<int64_t> reg_ids;
  std::vector<Reg*> regs;
  std::vector<std::vector<GateOp>> circuits;  // kept for re-planning (tuneBatch)
  int prec = QS_C64;
  Arith arith = Arith::F32;
  int k_req = 0;
  int max_ops = 0;  // cap on operations per fused pass (0 = the planner's default)
  // device data of the current plan
  FPass* d_passes = nullptr;
  FOp* d_ops = nullptr;
  FStage* d_st = nullptr;
  BItem* d_items = nullptr;
  BDep* d_deps = nullptr;     // persistent form: each pass's predecessor
  int* d_done = nullptr;      // persistent form: tiles done per pass, then the ticket
  bool persistent = false;
  bool diag_stall = false;    // every wait needs one tile too many (diagnostic)
  NormDesc* d_norms = nullptr;
  double* d_out = nullptr;
  double* h_out = nullptr;
  std::vector<Wave> waves;
  int64_t passes = 0;
  double bytes = 0, flops = 0, alu = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

std::mutex g_bmu;
std::unordered_map<int64_t, Batch*> g_batches;
int64_t g_next_batch = 1;

void free_plan(Batch& b) {
  if (b.exec) cudaGraphExecDestroy(b.exec);
  if (b.graph) cudaGraphDestroy(b.graph);
  cudaFree(b.d_passes);
  cudaFree(b.d_ops);
  cudaFree(b.d_st);
  cudaFree(b.d_items);
  cudaFree(b.d_deps);
  cudaFree(b.d_done);
  cudaFree(b.d_norms);
  cudaFree(b.d_out);
  if (b.h_out) cudaFreeHost(b.h_out);
  b.exec = nullptr;
  b.graph = nullptr;
  b.d_passes = nullptr;
  b.d_ops = nullptr;
  b.d_st = nullptr;
  b.d_items = nullptr;
  b.d_deps = nullptr;
  b.d_done = nullptr;
  b.d_norms = nullptr;
  b.d_out = nullptr;
  b.h_out = nullptr;
  b.waves.clear();
}

template <typename T>
T* upload(const std::vector<T>& v, cudaStream_t s) {
  T* d = nullptr;
  if (v.empty()) return d;
  QS_CUDA(cudaMalloc(&d, v.size() * sizeof(T)));
  QS_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return d;
}

template <class A, int R>
void launch_wave(const Batch& b, const Wave& w, cudaStream_t s) {
  const size_t smem = fused_smem_bytes<A>(w.kmax, w.Lmin, w.opmax, w.stmax);
  const int64_t chunks = (w.nitems + kBatchChunk - 1) / kBatchChunk;
  const int grid = int(std::min<int64_t>(chunks, int64_t(b.env->sms) * fused_ctas_per_sm(R)));
  k_fused_batch<A, R><<<grid, kFusedThreads, smem, s>>>(b.d_items + w.first_item, w.nitems, b.d_passes,
                                                        b.d_ops, b.d_st, w.kmax, w.Lmin, w.opmax);
}

// Every wave in one launch: CTAs claim item runs in list order and wait
// (bounded) for a register's previous pass (k_fused_batch_persist).
template <class A, int R>
void launch_persistent(const Batch& b, int nitems, int kmax, int Lmin, int opmax, int stmax, cudaStream_t s) {
  const size_t smem = fused_smem_bytes<A>(kmax, Lmin, opmax, stmax);
  const int64_t chunks = (nitems + kBatchChunk - 1) / kBatchChunk;
  const int grid = int(std::min<int64_t>(chunks, int64_t(b.env->sms) * fused_ctas_per_sm(R)));
  const int npass = int(b.passes);
  k_fused_batch_persist<A, R><<<grid, kFusedThreads, smem, s>>>(
      b.d_items, nitems, b.d_passes, b.d_ops, b.d_st, b.d_deps, b.d_done,
      reinterpret_cast<unsigned*>(b.d_done + npass), b.env->d_status, kmax, Lmin, opmax,
      b.diag_stall ? 2000000ull : 1000000000ull);
}

template <class A, int R>
void set_batch_attr() {
  // once per instantiation (thread-safe static initialisation)
  static const bool done = [] {
    QS_CUDA(cudaFuncSetAttribute(k_fused_batch<A, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 110 * 1024));
    QS_CUDA(cudaFuncSetAttribute(k_fused_batch_persist<A, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 110 * 1024));
    return true;
  }();
  (void)done;
}

// Plans every register with tile size k_req, uploads, captures the graph.
void build(Batch& b) {
  free_plan(b);
  Env& env = *b.env;
  std::vector<RegPlan> plans(b.regs.size());
  size_t maxp = 0;
  // the batch's own fusion depth for its plans (the env's option otherwise)
  struct DepthScope {
    Env& e;
    int64_t saved;
    DepthScope(Env& env_, int64_t d) : e(env_), saved(env_.max_fused_ops) { e.max_fused_ops = d; }
    ~DepthScope() { e.max_fused_ops = saved; }
  } depth_scope(env, b.max_ops > 0 ? b.max_ops : env.max_fused_ops);
  // k_fused_batch runs every tile on one CTA with a fixed number of register
  // bits per stage, so the batch's plans never spread a single-tile register
  // over a thread-block cluster (whose plans take fewer register bits)
  struct ClusterScope {
    Env& e;
    int64_t saved;
    explicit ClusterScope(Env& env_) : e(env_), saved(env_.fused_cluster) { e.fused_cluster = 0; }
    ~ClusterScope() { e.fused_cluster = saved; }
  } cluster_scope(env);
  const int kernel_R = b.arith == Arith::F32 ? 5 : 4;
  for (size_t r = 0; r < b.regs.size(); ++r) {
    // every replay starts from |0...0> (the first pass generates it)
    const int nq = b.regs[r]->nq;
    build_plan(*b.regs[r], b.circuits[r], b.k_req, nq >= 64 ? ~uint64_t(0) : (uint64_t(1) << nq) - 1,
               1.0, plans[r]);
    b.regs[r]->zero_bits = 0;  // the register's contents are the batch's from now on
    b.regs[r]->pend_scale = 1.0;
    b.regs[r]->reset_qscale();
    if (plans[r].R != kernel_R || plans[r].cluster > 1)
      fail(QS_E_ARG, "batch plan with " + std::to_string(plans[r].R) + " register bits (kernel takes " +
                         std::to_string(kernel_R) + ")");
    if (!plans[r].fps.empty()) plans[r].fps[0].init = 1;
    maxp = std::max(maxp, plans[r].fps.size());
  }
  // concatenate, rebasing op / stage indices
  std::vector<FPass> passes;
  std::vector<FOp> ops;
  std::vector<FStage> st;
  std::vector<std::vector<int>> pass_index(b.regs.size());
  b.passes = 0;
  b.bytes = 0;
  b.flops = 0;
  b.alu = 0;
  for (size_t r = 0; r < b.regs.size(); ++r) {
    const RegPlan& pl = plans[r];
    const int op0 = int(ops.size()), st0 = int(st.size());
    ops.insert(ops.end(), pl.fops.begin(), pl.fops.end());
    st.insert(st.end(), pl.fst.begin(), pl.fst.end());
    for (size_t p = 0; p < pl.fps.size(); ++p) {
      FPass fp = pl.fps[p];
      fp.op_begin += op0;
      fp.stage_begin += st0;
      fp.stage_end += st0;
      pass_index[r].push_back(int(passes.size()));
      passes.push_back(fp);
    }
    b.passes += int64_t(pl.fps.size());
  }
  // waves: big tiles first within a wave (they dominate the time)
  std::vector<BItem> items;
  const double S = b.prec == QS_C128 ? 16.0 : 8.0;
  for (size_t w = 0; w < maxp; ++w) {
    Wave wave;
    wave.first_item = int(items.size());
    std::vector<size_t> order;
    for (size_t r = 0; r < b.regs.size(); ++r)
      if (pass_index[r].size() > w) order.push_back(r);
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t x, size_t y) { return plans[x].k > plans[y].k; });
    for (size_t r : order) {
      const int pi = pass_index[r][w];
      const FPass& fp = passes[pi];
      for (int64_t t = 0; t < fp.ntiles; ++t) items.push_back(BItem{pi, 0, t});
      wave.kmax = std::max(wave.kmax, fp.k);
      wave.Lmin = std::min(wave.Lmin, fp.L);
      wave.opmax = std::max(wave.opmax, fp.op_count);
      wave.stmax = std::max(wave.stmax, fp.stage_end - fp.stage_begin);
      const double amps = std::ldexp(1.0, fp.nq);
      wave.bytes += amps * S * (fp.init ? 1.0 : 2.0);
      wave.flops += plans[r].flops[w];
      wave.alu += plans[r].alu[w];
    }
    wave.nitems = int(items.size()) - wave.first_item;
    b.bytes += wave.bytes;
    b.flops += wave.flops;
    b.alu += wave.alu;
    b.waves.push_back(wave);
  }
  // predecessor of every pass (persistent form): the register's previous pass
  std::vector<BDep> deps(passes.size(), BDep{-1, 0});
  for (size_t r = 0; r < b.regs.size(); ++r)
    for (size_t w = 1; w < pass_index[r].size(); ++w) {
      const int prev = pass_index[r][w - 1];
      deps[size_t(pass_index[r][w])] =
          BDep{prev, int(passes[size_t(prev)].ntiles) + (env.batch_diag_stall ? 1 : 0)};
    }
  std::vector<NormDesc> nd;
  for (Reg* r : b.regs) {
    nd.push_back(NormDesc{r->d, r->dim});
    b.bytes += double(r->dim) * S;
  }
  cudaStream_t s = env.stream;
  b.d_passes = upload(passes, s);
  b.d_ops = upload(ops, s);
  b.d_st = upload(st, s);
  b.d_items = upload(items, s);
  b.d_norms = upload(nd, s);
  b.persistent = env.batch_persistent != 0;
  b.diag_stall = env.batch_diag_stall != 0;
  if (b.persistent) {
    b.d_deps = upload(deps, s);
    QS_CUDA(cudaMalloc(&b.d_done, sizeof(int) * (passes.size() + 1)));
  }
  QS_CUDA(cudaMalloc(&b.d_out, sizeof(double) * b.regs.size()));
  QS_CUDA(cudaMallocHost(&b.h_out, sizeof(double) * b.regs.size()));
  QS_CUDA(cudaStreamSynchronize(s));
  if (b.arith == Arith::DF) set_batch_attr<DFArith, 4>();
  else if (b.arith == Arith::F64) set_batch_attr<PlainArith<double>, 4>();
  else set_batch_attr<PlainArith<float>, 5>();

  // capture: the waves, then the norms.  The first call that fails inside
  // the capture is named in the error (later ones only report the
  // invalidated capture).
  std::string first_err;
  auto note = [&](cudaError_t e, const std::string& what) {
    if (e != cudaSuccess && first_err.empty()) first_err = what + ": " + cudaGetErrorString(e);
  };
  QS_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  if (b.persistent) {
    int kmax = 0, Lmin = 64, opmax = 0, stmax = 0;
    for (const Wave& w : b.waves) {
      kmax = std::max(kmax, w.kmax);
      Lmin = std::min(Lmin, w.Lmin);
      opmax = std::max(opmax, w.opmax);
      stmax = std::max(stmax, w.stmax);
    }
    const int nitems = int(items.size());
    note(cudaMemsetAsync(b.d_done, 0, sizeof(int) * (passes.size() + 1), s), "clearing the pass counters");
    if (nitems == 0) {
      // registers with no queued gates: nothing to launch (as with no waves)
    } else if (b.arith == Arith::DF) launch_persistent<DFArith, 4>(b, nitems, kmax, Lmin, opmax, stmax, s);
    else if (b.arith == Arith::F64) launch_persistent<PlainArith<double>, 4>(b, nitems, kmax, Lmin, opmax, stmax, s);
    else launch_persistent<PlainArith<float>, 5>(b, nitems, kmax, Lmin, opmax, stmax, s);
    note(cudaGetLastError(), "persistent launch (items " + std::to_string(nitems) + ", k " + std::to_string(kmax) +
                                 ", L " + std::to_string(Lmin) + ", ops " + std::to_string(opmax) + ", stages " +
                                 std::to_string(stmax) + ")");
  } else {
    for (size_t wi = 0; wi < b.waves.size(); ++wi) {
      const Wave& w = b.waves[wi];
      if (b.arith == Arith::DF) launch_wave<DFArith, 4>(b, w, s);
      else if (b.arith == Arith::F64) launch_wave<PlainArith<double>, 4>(b, w, s);
      else launch_wave<PlainArith<float>, 5>(b, w, s);
      note(cudaGetLastError(), "wave " + std::to_string(wi) + " launch (items " + std::to_string(w.nitems) +
                                   ", k " + std::to_string(w.kmax) + ", L " + std::to_string(w.Lmin) + ", ops " +
                                   std::to_string(w.opmax) + ", stages " + std::to_string(w.stmax) + ")");
    }
  }
  const int nreg = int(b.regs.size());
  if (b.prec == QS_C128) k_batch_norms<double2><<<nreg, kNormThreads, 0, s>>>(b.d_norms, b.d_out);
  else k_batch_norms<float2><<<nreg, kNormThreads, 0, s>>>(b.d_norms, b.d_out);
  note(cudaGetLastError(), "norms launch");
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(s, &g);
  if (!first_err.empty()) {
    if (g) cudaGraphDestroy(g);
    fail(QS_E_CUDA, "batch " + first_err);
  }
  if (ce != cudaSuccess) fail(QS_E_CUDA, std::string("batch capture: ") + cudaGetErrorString(ce));
  b.graph = g;
  QS_CUDA(cudaGraphInstantiate(&b.exec, b.graph, 0));
}

Batch& batch_of(QSBatch h) {
  std::lock_guard<std::mutex> lk(g_bmu);
  auto it = g_batches.find(h.id);
  if (it == g_batches.end()) fail(QS_E_HANDLE, "unknown batch handle " + std::to_string(h.id));
  return *it->second;
}

void run(Batch& b) {
  KTimer kt(*b.env, "batch_graph", b.bytes, b.flops, int(b.waves.size()) + 1, b.alu);
  QS_CUDA(cudaGraphLaunch(b.exec, b.env->stream));
}

}  // namespace

}  // namespace qs

using namespace qs;

extern "C" {

int createBatch(QuESTEnv e, const Qureg* regs, int count, int tileQubits, QSBatch* out) {
  return guarded_call([&] {
    if (!out || (count > 0 && !regs)) fail(QS_E_ARG, "null pointer");
    if (count < 1) fail(QS_E_ARG, "a batch needs at least one register");
    if (tileQubits != 0 && (tileQubits < 5 || tileQubits > 13)) fail(QS_E_ARG, "tileQubits must be 0 or 5..13");
    Env& env = lookup_env(e.id);
    auto* b = new Batch();
    b->env = &env;
    b->k_req = tileQubits;
    try {
      std::vector<int64_t> seen;
      for (int i = 0; i < count; ++i) {
        Reg& r = lookup_reg(regs[i].id);
        if (r.env != &env) fail(QS_E_ARG, "register of another environment");
        if (r.density) fail(QS_E_ARG, "batches hold state vectors");
        if (i == 0) b->prec = r.prec;
        if (r.prec != b->prec) fail(QS_E_ARG, "all registers of a batch share one precision");
        if (!fusable(r)) fail(QS_E_QUBIT, "register too small for a batch (needs >= 4 qubits for QS_C128, 5 for QS_C64)");
        if (std::find(seen.begin(), seen.end(), r.id) != seen.end()) fail(QS_E_DUP, "register listed twice");
        seen.push_back(r.id);
        b->regs.push_back(&r);
        b->reg_ids.push_back(r.id);
      }
      b->arith = arith_of(*b->regs[0]);
      for (Reg* r : b->regs)
        for (const GateOp& op : r->queue)
          if (op.k == OpK::MULTI) fail(QS_E_ARG, "batches take single-target gates only");
      for (Reg* r : b->regs) {
        b->circuits.push_back(r->queue);
        r->queue.clear();
      }
      const int64_t prof = env.profile;
      env.profile = 0;
      try {
        build(*b);
      } catch (...) {
        env.profile = prof;
        throw;
      }
      env.profile = prof;
    } catch (...) {
      free_plan(*b);
      delete b;
      throw;
    }
    std::lock_guard<std::mutex> lk(g_bmu);
    b->id = g_next_batch++;
    g_batches[b->id] = b;
    out->id = b->id;
  });
}

int runBatch(QSBatch h) {
  return guarded_call([&] {
    Batch& b = batch_of(h);
    for (Reg* r : b.regs) {
      r->zero_bits = 0;
      r->pend_scale = 1.0;
      r->reset_qscale();
    }
    run(b);
  });
}

int getBatchNorms(QSBatch h, double* out) {
  return guarded_call([&] {
    Batch& b = batch_of(h);
    if (!out) fail(QS_E_ARG, "null output");
    cudaStream_t s = b.env->stream;
    QS_CUDA(cudaMemcpyAsync(b.h_out, b.d_out, sizeof(double) * b.regs.size(), cudaMemcpyDeviceToHost, s));
    QS_CUDA(cudaMemcpyAsync(b.env->h_status, b.env->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    QS_CUDA(cudaStreamSynchronize(s));
    check_status(*b.env);  // a bounded wait of the persistent form that ran out
    std::memcpy(out, b.h_out, sizeof(double) * b.regs.size());
  });
}

int getBatchInfo(QSBatch h, int* tileQubits, int64_t* passes, int* waves, double* bytes, double* flops) {
  return guarded_call([&] {
    Batch& b = batch_of(h);
    if (tileQubits) *tileQubits = b.k_req;
    if (passes) *passes = b.passes;
    if (waves) *waves = int(b.waves.size());
    if (bytes) *bytes = b.bytes;
    if (flops) *flops = b.flops;
  });
}

int tuneBatch(QSBatch h, const int* candidates, int numCandidates, int replays, int* chosen) {
  return guarded_call([&] {
    Batch& b = batch_of(h);
    if (!candidates || numCandidates < 1) fail(QS_E_ARG, "no candidate tile sizes");
    if (replays < 1) fail(QS_E_ARG, "replays must be >= 1");
    for (int i = 0; i < numCandidates; ++i)
      if (candidates[i] < 5 || candidates[i] > 13) fail(QS_E_ARG, "candidate tile sizes must be 5..13");
    Env& env = *b.env;
    cudaEvent_t e0, e1;
    QS_CUDA(cudaEventCreate(&e0));
    QS_CUDA(cudaEventCreate(&e1));
    const int64_t prof = env.profile;
    env.profile = 0;
    float best = 1e30f;
    int best_k = b.k_req;
    try {
      for (int i = 0; i < numCandidates; ++i) {
        b.k_req = candidates[i];
        build(b);
        QS_CUDA(cudaGraphLaunch(b.exec, env.stream));  // warm-up
        QS_CUDA(cudaEventRecord(e0, env.stream));
        for (int r = 0; r < replays; ++r) QS_CUDA(cudaGraphLaunch(b.exec, env.stream));
        QS_CUDA(cudaEventRecord(e1, env.stream));
        QS_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        QS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
          best = ms;
          best_k = candidates[i];
        }
      }
      b.k_req = best_k;
      build(b);
    } catch (...) {
      env.profile = prof;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    env.profile = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (chosen) *chosen = best_k;
  });
}

int tuneBatchJoint(QSBatch h, const int* tileCandidates, int numTile, const int* depthCandidates, int numDepth,
                   int replays, int* chosenTile, int* chosenDepth) {
  return guarded_call([&] {
    Batch& b = batch_of(h);
    if (!tileCandidates || numTile < 1 || !depthCandidates || numDepth < 1)
      fail(QS_E_ARG, "no candidates");
    if (replays < 1) fail(QS_E_ARG, "replays must be >= 1");
    for (int i = 0; i < numTile; ++i)
      if (tileCandidates[i] < 5 || tileCandidates[i] > 13) fail(QS_E_ARG, "candidate tile sizes must be 5..13");
    for (int i = 0; i < numDepth; ++i)
      if (depthCandidates[i] < 0 || depthCandidates[i] > kMaxPassOps)
        fail(QS_E_ARG, "candidate depths must be 0 (default) or 1.." + std::to_string(kMaxPassOps));
    Env& env = *b.env;
    cudaEvent_t e0, e1;
    QS_CUDA(cudaEventCreate(&e0));
    QS_CUDA(cudaEventCreate(&e1));
    const int64_t prof = env.profile;
    env.profile = 0;
    float best = 1e30f;
    int best_k = b.k_req, best_d = b.max_ops;
    try {
      for (int i = 0; i < numTile; ++i) {
        for (int j = 0; j < numDepth; ++j) {
          b.k_req = tileCandidates[i];
          b.max_ops = depthCandidates[j];
          build(b);
          QS_CUDA(cudaGraphLaunch(b.exec, env.stream));  // warm-up
          QS_CUDA(cudaEventRecord(e0, env.stream));
          for (int r = 0; r < replays; ++r) QS_CUDA(cudaGraphLaunch(b.exec, env.stream));
          QS_CUDA(cudaEventRecord(e1, env.stream));
          QS_CUDA(cudaEventSynchronize(e1));
          float ms = 0;
          QS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          if (ms < best) {
            best = ms;
            best_k = b.k_req;
            best_d = b.max_ops;
          }
        }
      }
      b.k_req = best_k;
      b.max_ops = best_d;
      build(b);
    } catch (...) {
      env.profile = prof;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    env.profile = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (chosenTile) *chosenTile = best_k;
    if (chosenDepth) *chosenDepth = best_d;
  });
}

int destroyBatch(QSBatch h) {
  return guarded_call([&] {
    Batch& b = batch_of(h);
    cudaStreamSynchronize(b.env->stream);
    free_plan(b);
    std::lock_guard<std::mutex> lk(g_bmu);
    g_batches.erase(b.id);
    delete &b;
  });
}

}  // extern "C"
