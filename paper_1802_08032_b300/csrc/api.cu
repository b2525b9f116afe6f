// C-ABI entry points (declared in qsim.h): handle tables, argument
// validation, register memory, and dispatch to the kernel layer.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "jit_runtime.h"
#include "runtime.h"

using namespace qs;

namespace {

thread_local std::string t_err;
std::mutex g_mu;
std::unordered_map<int64_t, Env*> g_envs;
std::unordered_map<int64_t, Reg*> g_regs;
int64_t g_next_id = 1;

template <class F>
int guarded(F&& f) {
  try {
    f();
    return QS_OK;
  } catch (const Error& e) {
    t_err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    t_err = "host allocation failed";
    return QS_E_NOMEM;
  } catch (const std::exception& e) {
    t_err = e.what();
    return QS_E_ARG;
  }
}

Env& env_of(QuESTEnv e) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_envs.find(e.id);
  if (it == g_envs.end()) fail(QS_E_HANDLE, "unknown environment handle " + std::to_string(e.id));
  return *it->second;
}

Reg& reg_of(Qureg q) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_regs.find(q.id);
  if (it == g_regs.end()) fail(QS_E_HANDLE, "unknown register handle " + std::to_string(q.id));
  return *it->second;
}

void need(const void* p, const char* what) {
  if (!p) fail(QS_E_ARG, std::string("null pointer: ") + what);
}

void apply(Reg& r, const GateOp& op) {
  if (r.env->fusion) {
    r.queue.push_back(op);
  } else {
    launch_op(*r.env, r, op);
    note_mixing(r, op);
  }
}

void* dev_alloc(Env& env, size_t bytes) {
  if (env.budget > 0 && env.used + int64_t(bytes) > env.budget)
    fail(QS_E_NOMEM, "memory budget exceeded: " + std::to_string(env.used + bytes) + " > " +
                         std::to_string(env.budget) + " bytes");
  void* p = nullptr;
  if (env.alloc) {
    p = env.alloc(bytes, env.actx);
    if (!p) fail(QS_E_NOMEM, "allocator hook returned null for " + std::to_string(bytes) + " bytes");
  } else {
    const cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(QS_E_NOMEM, "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
  }
  env.used += int64_t(bytes);
  return p;
}

void dev_free(Env& env, void* p, size_t bytes) {
  if (!p) return;
  if (env.release) env.release(p, env.actx);
  else cudaFree(p);
  env.used -= int64_t(bytes);
}

void ensure_stage(Env& env) {
  if (env.d_stage) return;
  env.stage_amps = int64_t(1) << 22;  // 64 MiB of double2
  QS_CUDA(cudaMalloc(&env.d_stage, size_t(env.stage_amps) * sizeof(double2)));
}

void init_zero(Reg& r) {
  r.queue.clear();
  r.pend_scale = 1.0;
  r.reset_qscale();
  r.zero_bits = r.nq >= 64 ? ~uint64_t(0) : (uint64_t(1) << r.nq) - 1;
  const size_t amp = r.prec == QS_C128 ? sizeof(double2) : sizeof(float2);
  QS_CUDA(cudaMemsetAsync(r.d, 0, size_t(r.dim) * amp, r.env->stream));
  if (r.prec == QS_C128) {
    static const double one[2] = {1.0, 0.0};
    QS_CUDA(cudaMemcpyAsync(r.d, one, sizeof(one), cudaMemcpyHostToDevice, r.env->stream));
  } else {
    static const float one[2] = {1.0f, 0.0f};
    QS_CUDA(cudaMemcpyAsync(r.d, one, sizeof(one), cudaMemcpyHostToDevice, r.env->stream));
  }
}

int create_reg(int n, int prec, QuESTEnv e, Qureg* out, bool density) {
  return guarded([&] {
    need(out, "out");
    Env& env = env_of(e);
    if (prec != QS_C64 && prec != QS_C128) fail(QS_E_ARG, "precision must be QS_C64 or QS_C128");
    const int nq = density ? 2 * n : n;
    if (n < 1 || nq > 40) fail(QS_E_QUBIT, "unsupported qubit count " + std::to_string(n));
    QS_CUDA(cudaSetDevice(env.device));
    auto* r = new Reg();
    r->env = &env;
    r->n = n;
    r->density = density;
    r->nq = nq;
    r->prec = prec;
    r->dim = int64_t(1) << nq;
    r->bytes = size_t(r->dim) * (prec == QS_C128 ? 16 : 8);
    try {
      r->d = dev_alloc(env, r->bytes);
      init_zero(*r);
    } catch (...) {
      if (r->d) dev_free(env, r->d, r->bytes);
      delete r;
      throw;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    r->id = g_next_id++;
    g_regs[r->id] = r;
    env.regs.push_back(r->id);
    out->id = r->id;
  });
}

void destroy_reg_locked(Reg* r) {
  Env& env = *r->env;
  cudaStreamSynchronize(env.stream);
  dev_free(env, r->d, r->bytes);
  env.regs.erase(std::remove(env.regs.begin(), env.regs.end(), r->id), env.regs.end());
  delete r;
}

int one_op(Qureg q, const QSOp& o) {
  return guarded([&] {
    Reg& r = reg_of(q);
    std::vector<GateOp> ops;
    convert_op(r, o, ops);
    for (auto& op : ops) apply(r, op);
  });
}

QSOp blank(int kind, int target) {
  QSOp o;
  std::memset(&o, 0, sizeof(o));
  o.kind = kind;
  o.target = target;
  return o;
}

void mat_params(const ComplexMatrix2& u, double* p) {
  for (int rr = 0; rr < 2; ++rr)
    for (int cc = 0; cc < 2; ++cc) {
      p[2 * (2 * rr + cc)] = u.m[rr][cc].re;
      p[2 * (2 * rr + cc) + 1] = u.m[rr][cc].im;
    }
}

}  // namespace

namespace qs {
void set_last_error(const std::string& msg) { t_err = msg; }
int guarded_call(const std::function<void()>& f) { return guarded(f); }
Env& lookup_env(int64_t id) { return env_of(QuESTEnv{id}); }
Reg& lookup_reg(int64_t id) { return reg_of(Qureg{id}); }
void apply_op(Reg& r, const GateOp& op) { apply(r, op); }
}

extern "C" {

const char* qsLastError(void) { return t_err.c_str(); }

int createQuESTEnv(QuESTEnv* out) {
  return guarded([&] {
    need(out, "out");
    auto* env = new Env();
    try {
      QS_CUDA(cudaGetDevice(&env->device));
      QS_CUDA(cudaDeviceGetAttribute(&env->sms, cudaDevAttrMultiProcessorCount, env->device));
      QS_CUDA(cudaStreamCreateWithFlags(&env->own, cudaStreamNonBlocking));
      env->stream = env->own;
      QS_CUDA(cudaMalloc(&env->d_partial, sizeof(double) * 4096));
      QS_CUDA(cudaMalloc(&env->d_result, sizeof(double) * 64));
      QS_CUDA(cudaMallocHost(&env->h_result, sizeof(double) * 64));
      QS_CUDA(cudaMalloc(&env->d_status, sizeof(unsigned)));
      QS_CUDA(cudaMemset(env->d_status, 0, sizeof(unsigned)));
      QS_CUDA(cudaMallocHost(&env->h_status, sizeof(unsigned)));
      *env->h_status = 0;
    } catch (...) {
      if (env->own) cudaStreamDestroy(env->own);
      if (env->d_partial) cudaFree(env->d_partial);
      if (env->d_result) cudaFree(env->d_result);
      if (env->h_result) cudaFreeHost(env->h_result);
      if (env->d_status) cudaFree(env->d_status);
      delete env;
      throw;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    env->id = g_next_id++;
    g_envs[env->id] = env;
    out->id = env->id;
  });
}

int destroyQuESTEnv(QuESTEnv e) {
  return guarded([&] {
    Env& env = env_of(e);
    cudaStreamSynchronize(env.stream);
    std::lock_guard<std::mutex> lk(g_mu);
    for (int64_t id : std::vector<int64_t>(env.regs)) {
      auto it = g_regs.find(id);
      if (it != g_regs.end()) {
        destroy_reg_locked(it->second);
        g_regs.erase(it);
      }
    }
    env.prof.reset();
    for (cudaEvent_t ev : env.prof.pool) cudaEventDestroy(ev);
    free_fused_buffers(env);
    cudaFree(env.d_partial);
    cudaFree(env.d_result);
    cudaFreeHost(env.h_result);
    cudaFree(env.d_status);
    cudaFreeHost(env.h_status);
    if (env.d_stage) cudaFree(env.d_stage);
    cudaStreamDestroy(env.own);
    g_envs.erase(env.id);
    delete &env;
    // the last environment: no background compile may outlive the library's
    // users (a compile running while the process exits can crash it)
    if (g_envs.empty()) jit_shutdown();
  });
}

int qsJitShutdown(void) {
  return guarded([&] { jit_shutdown(); });
}

int syncQuESTEnv(QuESTEnv e) {
  return guarded([&] {
    Env& env = env_of(e);
    std::vector<Reg*> regs;
    {
      std::lock_guard<std::mutex> lk(g_mu);
      for (int64_t id : env.regs) regs.push_back(g_regs.at(id));
    }
    for (Reg* r : regs) flush(*r);
    QS_CUDA(cudaMemcpyAsync(env.h_status, env.d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, env.stream));
    QS_CUDA(cudaStreamSynchronize(env.stream));
    QS_CUDA(cudaGetLastError());
    check_status(env);
  });
}

int qsDiagBoundedWait(QuESTEnv e, int timeoutUs) {
  return guarded([&] {
    Env& env = env_of(e);
    if (timeoutUs < 1 || timeoutUs > 1000000) fail(QS_E_ARG, "timeoutUs must be in 1..1000000");
    launch_wait_probe(env, timeoutUs);
  });
}

int setEnvOption(QuESTEnv e, const char* key, int64_t value) {
  return guarded([&] {
    Env& env = env_of(e);
    need(key, "key");
    const std::string k(key);
    if (k == "fusion") {
      if (value != 0 && value != 1) fail(QS_E_ARG, "fusion must be 0 or 1");
      if (!value) {
        std::lock_guard<std::mutex> lk(g_mu);
        for (int64_t id : env.regs) flush(*g_regs.at(id));
      }
      env.fusion = value;
    } else if (k == "tile_qubits") {
      if (value != 0 && (value < 5 || value > 13)) fail(QS_E_ARG, "tile_qubits must be 0 or 5..13");
      env.tile_qubits = value;
    } else if (k == "max_fused_ops") {
      if (value < 0) fail(QS_E_ARG, "max_fused_ops must be >= 0");
      env.max_fused_ops = value;
    } else if (k == "budget_bytes") {
      if (value < 0) fail(QS_E_ARG, "budget_bytes must be >= 0");
      env.budget = value;
    } else if (k == "arith") {
      if (value != 0 && value != 1) fail(QS_E_ARG, "arith must be 0 (FP64) or 1 (double-float)");
      {
        std::lock_guard<std::mutex> lk(g_mu);
        for (int64_t id : env.regs) flush(*g_regs.at(id));
      }
      env.arith = value;
    } else if (k == "profile") {
      if (value != 0 && value != 1) fail(QS_E_ARG, "profile must be 0 or 1");
      env.profile = value;
    } else if (k == "fused_cluster") {
      if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8)
        fail(QS_E_ARG, "fused_cluster must be 0, 1, 2, 4 or 8");
      env.fused_cluster = value;
    } else if (k == "tile_low_qubits") {
      if (value != 0 && (value < 2 || value > 6)) fail(QS_E_ARG, "tile_low_qubits must be 0 (default) or 2..6");
      env.tile_low_qubits = value;
    } else if (k == "batch_persistent") {
      if (value != 0 && value != 1) fail(QS_E_ARG, "batch_persistent must be 0 or 1");
      env.batch_persistent = value;
    } else if (k == "batch_diag_stall") {
      if (value != 0 && value != 1) fail(QS_E_ARG, "batch_diag_stall must be 0 or 1");
      env.batch_diag_stall = value;
    } else if (k == "multi_tc_stage") {
      if (value != 0 && value != 1) fail(QS_E_ARG, "multi_tc_stage must be 0 or 1");
      env.multi_tc_stage = value;
    } else if (k == "multi_tc") {
      if (value < 0 || value > 2) fail(QS_E_ARG, "multi_tc must be 0, 1 or 2");
      env.multi_tc = value;
    } else if (k == "jit") {
      if (value < 0 || value > 2) fail(QS_E_ARG, "jit must be 0 (off), 1 (compile and wait) or 2 (background)");
      env.jit = value;
    } else if (k == "jit_min_qubits") {
      if (value < 1 || value > 64) fail(QS_E_ARG, "jit_min_qubits must be in 1..64");
      env.jit_min_qubits = value;
    } else if (k == "plan_cache") {
      if (value != 0 && value != 1) fail(QS_E_ARG, "plan_cache must be 0 or 1");
      env.plan_cache_on = value;
      if (!value) env.plan_cache.reset();
    } else if (k == "jit_copy") {
      if (value < -1 || value > 2)
        fail(QS_E_ARG, "jit_copy must be -1 (by arithmetic), 0 (plain), 1 (bulk) or 2 (async)");
      env.jit_copy = value;
    } else if (k == "jit_swizzle") {
      if (value != 0 && value != 1) fail(QS_E_ARG, "jit_swizzle must be 0 or 1");
      env.jit_swizzle = value;
    } else if (k == "jit_direct") {
      if (value != 0 && value != 1) fail(QS_E_ARG, "jit_direct must be 0 or 1");
      env.jit_direct = value;
    } else if (k == "jit_fp64") {
      if (value != 0 && value != 1) fail(QS_E_ARG, "jit_fp64 must be 0 or 1");
      env.jit_fp64 = value;
    } else if (k == "jit_ctas") {
      if (value < 0 || value > 4) fail(QS_E_ARG, "jit_ctas must be 0 (by shape) or 1..4");
      env.jit_ctas = value;
    } else {
      fail(QS_E_ARG, "unknown option " + k);
    }
  });
}

int getEnvOption(QuESTEnv e, const char* key, int64_t* value) {
  return guarded([&] {
    Env& env = env_of(e);
    need(key, "key");
    need(value, "value");
    const std::string k(key);
    if (k == "fusion") *value = env.fusion;
    else if (k == "tile_qubits") *value = env.tile_qubits;
    else if (k == "max_fused_ops") *value = env.max_fused_ops;
    else if (k == "budget_bytes") *value = env.budget;
    else if (k == "used_bytes") *value = env.used;
    else if (k == "profile") *value = env.profile;
    else if (k == "arith") *value = env.arith;
    else if (k == "multi_tc") *value = env.multi_tc;
    else if (k == "multi_tc_stage") *value = env.multi_tc_stage;
    else if (k == "fused_cluster") *value = env.fused_cluster;
    else if (k == "batch_persistent") *value = env.batch_persistent;
    else if (k == "tile_low_qubits") *value = env.tile_low_qubits;
    else if (k == "batch_diag_stall") *value = env.batch_diag_stall;
    else if (k == "jit") *value = env.jit;
    else if (k == "jit_min_qubits") *value = env.jit_min_qubits;
    else if (k == "jit_ctas") *value = env.jit_ctas;
    else if (k == "jit_fp64") *value = env.jit_fp64;
    else if (k == "jit_copy") *value = env.jit_copy;
    else if (k == "jit_direct") *value = env.jit_direct;
    else if (k == "jit_swizzle") *value = env.jit_swizzle;
    else if (k == "plan_cache") *value = env.plan_cache_on;
    else if (k == "plan_cache_hits") *value = env.plan_cache_hits;
    else if (k == "jit_launches") *value = env.jit_launches;
    else if (k == "jit_rejected") *value = env.jit_rejected;
    else if (k == "jit_ready") *value = jit_stats().ready;
    else if (k == "jit_pending") *value = jit_stats().pending;
    else if (k == "jit_failed") *value = jit_stats().failed;
    else if (k == "jit_compile_ms") *value = int64_t(jit_stats().compile_s * 1e3);
    else if (k == "launches") *value = env.launches;
    else if (k == "fused_passes") *value = env.fused_passes;
    else if (k == "fused_vops") *value = env.fused_vops;
    else fail(QS_E_ARG, "unknown option " + k);
  });
}

int setAllocator(QuESTEnv e, void* (*alloc)(size_t, void*), void (*release)(void*, void*), void* ctx) {
  return guarded([&] {
    Env& env = env_of(e);
    if ((alloc == nullptr) != (release == nullptr))
      fail(QS_E_ARG, "alloc and release must both be set or both be null");
    env.alloc = alloc;
    env.release = release;
    env.actx = ctx;
  });
}

int setStream(QuESTEnv e, void* stream) {
  return guarded([&] {
    Env& env = env_of(e);
    {
      std::lock_guard<std::mutex> lk(g_mu);
      for (int64_t id : env.regs) flush(*g_regs.at(id));
    }
    cudaStream_t next = stream ? static_cast<cudaStream_t>(stream) : env.own;
    if (next != env.stream) {
      // order the new stream after everything queued on the old one
      cudaEvent_t ev;
      QS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      QS_CUDA(cudaEventRecord(ev, env.stream));
      QS_CUDA(cudaStreamWaitEvent(next, ev, 0));
      QS_CUDA(cudaEventDestroy(ev));
    }
    env.stream = next;
  });
}

int createQureg(int n, int prec, QuESTEnv e, Qureg* out) { return create_reg(n, prec, e, out, false); }
int createDensityQureg(int n, int prec, QuESTEnv e, Qureg* out) { return create_reg(n, prec, e, out, true); }

int destroyQureg(Qureg q) {
  return guarded([&] {
    Reg& r = reg_of(q);
    std::lock_guard<std::mutex> lk(g_mu);
    g_regs.erase(r.id);
    destroy_reg_locked(&r);
  });
}

int initZeroState(Qureg q) {
  return guarded([&] { init_zero(reg_of(q)); });
}

int initPlusState(Qureg q) {
  return guarded([&] {
    Reg& r = reg_of(q);
    r.queue.clear();
    // |+>^n: every amplitude 2^(-n/2); |+><+|^N: every entry 2^(-N).
    const double v = r.density ? std::ldexp(1.0, -r.n) : 1.0 / std::sqrt(double(r.dim));
    launch_fill(*r.env, r, v, 0.0);
    r.zero_bits = 0;
    r.pend_scale = 1.0;
    r.reset_qscale();
  });
}

int copyStateToHost(Qureg q, Complex* dst, int64_t start, int64_t count) {
  return guarded([&] {
    Reg& r = reg_of(q);
    if (count == 0) return;
    need(dst, "dst");
    if (start < 0 || count < 0 || start > r.dim || count > r.dim - start)
      fail(QS_E_ARG, "amplitude range out of bounds");
    flush(r);
    Env& env = *r.env;
    if (r.prec == QS_C128) {
      QS_CUDA(cudaMemcpyAsync(dst, static_cast<double2*>(r.d) + start, size_t(count) * 16,
                              cudaMemcpyDeviceToHost, env.stream));
      QS_CUDA(cudaStreamSynchronize(env.stream));
      return;
    }
    ensure_stage(env);
    for (int64_t off = 0; off < count; off += env.stage_amps) {
      const int64_t c = std::min(env.stage_amps, count - off);
      launch_convert(env, static_cast<float2*>(r.d) + start + off, env.d_stage, c, true);
      QS_CUDA(cudaMemcpyAsync(dst + off, env.d_stage, size_t(c) * 16, cudaMemcpyDeviceToHost, env.stream));
      QS_CUDA(cudaStreamSynchronize(env.stream));
    }
  });
}

int setAmps(Qureg q, const Complex* src, int64_t start, int64_t count) {
  return guarded([&] {
    Reg& r = reg_of(q);
    if (count == 0) return;
    need(src, "src");
    if (start < 0 || count < 0 || start > r.dim || count > r.dim - start)
      fail(QS_E_ARG, "amplitude range out of bounds");
    flush(r);
    r.zero_bits = 0;
    Env& env = *r.env;
    if (r.prec == QS_C128) {
      QS_CUDA(cudaMemcpyAsync(static_cast<double2*>(r.d) + start, src, size_t(count) * 16,
                              cudaMemcpyHostToDevice, env.stream));
      QS_CUDA(cudaStreamSynchronize(env.stream));
      return;
    }
    ensure_stage(env);
    for (int64_t off = 0; off < count; off += env.stage_amps) {
      const int64_t c = std::min(env.stage_amps, count - off);
      QS_CUDA(cudaMemcpyAsync(env.d_stage, src + off, size_t(c) * 16, cudaMemcpyHostToDevice, env.stream));
      launch_convert(env, env.d_stage, static_cast<float2*>(r.d) + start + off, c, false);
      QS_CUDA(cudaStreamSynchronize(env.stream));
    }
  });
}

int getNumQubits(Qureg q, int* out) {
  return guarded([&] {
    need(out, "out");
    *out = reg_of(q).n;
  });
}

int getNumAmps(Qureg q, int64_t* out) {
  return guarded([&] {
    need(out, "out");
    *out = reg_of(q).dim;
  });
}

int getQuregInfo(Qureg q, int* numQubits, int* isDensity, int* precision, void** devicePtr) {
  return guarded([&] {
    Reg& r = reg_of(q);
    if (numQubits) *numQubits = r.n;
    if (isDensity) *isDensity = r.density ? 1 : 0;
    if (precision) *precision = r.prec;
    if (devicePtr) {
      flush(r);  // the amplitudes as stored must be the register's values
      *devicePtr = r.d;
      r.zero_bits = 0;  // the caller may write the amplitudes
    }
  });
}

int hadamard(Qureg q, int t) { return one_op(q, blank(QS_OP_H, t)); }
int pauliX(Qureg q, int t) { return one_op(q, blank(QS_OP_X, t)); }
int sqrtX(Qureg q, int t) { return one_op(q, blank(QS_OP_SQRTX, t)); }
int sqrtY(Qureg q, int t) { return one_op(q, blank(QS_OP_SQRTY, t)); }
int tGate(Qureg q, int t) { return one_op(q, blank(QS_OP_T, t)); }

int phaseShift(Qureg q, int t, double angle) {
  QSOp o = blank(QS_OP_PHASE, t);
  o.params[0] = angle;
  return one_op(q, o);
}

int compactUnitary(Qureg q, int t, Complex alpha, Complex beta) {
  QSOp o = blank(QS_OP_COMPACT, t);
  o.params[0] = alpha.re;
  o.params[1] = alpha.im;
  o.params[2] = beta.re;
  o.params[3] = beta.im;
  return one_op(q, o);
}

int unitary(Qureg q, int t, ComplexMatrix2 u) {
  QSOp o = blank(QS_OP_UNITARY, t);
  mat_params(u, o.params);
  return one_op(q, o);
}

int controlledNot(Qureg q, int c, int t) {
  QSOp o = blank(QS_OP_CNOT, t);
  o.numControls = 1;
  o.controls[0] = c;
  return one_op(q, o);
}

int controlledUnitary(Qureg q, int c, int t, ComplexMatrix2 u) {
  QSOp o = blank(QS_OP_CUNITARY, t);
  o.numControls = 1;
  o.controls[0] = c;
  mat_params(u, o.params);
  return one_op(q, o);
}

int multiControlledUnitary(Qureg q, const int* ctrls, int nc, int t, ComplexMatrix2 u) {
  return guarded([&] {
    Reg& r = reg_of(q);
    if (nc < 0 || nc >= r.n) fail(QS_E_ARG, "numControls out of range");
    if (nc > 0) need(ctrls, "controls");
    const uint64_t cm = check_targets(r, t, ctrls, nc);
    double p[8];
    mat_params(u, p);
    check_unitary(p);
    GateOp op = make_op(OpK::GEN, t, cm);
    std::memcpy(op.m, p, sizeof(p));
    apply(r, op);
  });
}

int multiControlledMultiQubitUnitary(Qureg q, const int* ctrls, int nc, const int* targets, int nt,
                                     const Complex* u) {
  return guarded([&] {
    Reg& r = reg_of(q);
    if (nt < 1 || nt > 5) fail(QS_E_ARG, "numTargets must be in 1..5");
    need(targets, "targets");
    need(u, "matrix");
    if (nc < 0 || nc > r.n - nt) fail(QS_E_ARG, "numControls out of range");
    if (nc > 0) need(ctrls, "controls");
    uint64_t tmask = 0;
    for (int k = 0; k < nt; ++k) {
      check_qubit(r, targets[k], "target");
      const uint64_t b = uint64_t(1) << targets[k];
      if (tmask & b) fail(QS_E_DUP, "target " + std::to_string(targets[k]) + " repeated");
      tmask |= b;
    }
    uint64_t cmask = 0;
    for (int k = 0; k < nc; ++k) {
      check_qubit(r, ctrls[k], "control");
      const uint64_t b = uint64_t(1) << ctrls[k];
      if ((cmask | tmask) & b) fail(QS_E_DUP, "qubit " + std::to_string(ctrls[k]) + " repeated among targets and controls");
      cmask |= b;
    }
    const int d = 1 << nt;
    auto mat = std::make_shared<std::vector<double>>(size_t(2 * d * d));
    for (int e = 0; e < d * d; ++e) {
      (*mat)[2 * e] = u[e].re;
      (*mat)[2 * e + 1] = u[e].im;
    }
    // max |U U^dagger - I| <= 1e-10
    double worst = 0;
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        double re = 0, im = 0;
        for (int s = 0; s < d; ++s) {
          const double ar = u[i * d + s].re, ai = u[i * d + s].im;
          const double br = u[j * d + s].re, bi = -u[j * d + s].im;
          re += ar * br - ai * bi;
          im += ar * bi + ai * br;
        }
        worst = std::max(worst, std::hypot(re - (i == j ? 1.0 : 0.0), im));
      }
    if (!(worst <= 1e-10))
      fail(QS_E_UNITARY, "matrix is not unitary (max |UU^dagger - I| = " + std::to_string(worst) + ")");
    GateOp op = make_op(OpK::MULTI, targets[0], cmask);
    op.nt = nt;
    for (int k = 0; k < nt; ++k) op.tg[k] = uint8_t(targets[k]);
    op.big = mat;
    apply(r, op);
  });
}

int multiQubitUnitary(Qureg q, const int* targets, int nt, const Complex* u) {
  return multiControlledMultiQubitUnitary(q, nullptr, 0, targets, nt, u);
}

int twoQubitUnitary(Qureg q, int t1, int t2, ComplexMatrix4 u) {
  const int t[2] = {t1, t2};
  return multiControlledMultiQubitUnitary(q, nullptr, 0, t, 2, &u.m[0][0]);
}

int controlledPhaseFlip(Qureg q, int a, int b) {
  QSOp o = blank(QS_OP_CZ, a);
  o.target2 = b;
  return one_op(q, o);
}

int multiControlledPhaseFlip(Qureg q, const int* ctrls, int nc) {
  return guarded([&] {
    Reg& r = reg_of(q);
    if (nc < 1 || nc > r.n) fail(QS_E_ARG, "numControls must be in [1, numQubits]");
    need(ctrls, "controls");
    const uint64_t cm = check_targets(r, -1, ctrls, nc);
    apply(r, make_op(OpK::SIGN, -1, cm));
  });
}

int mixDephasing(Qureg q, int t, double p) {
  QSOp o = blank(QS_OP_DEPHASE, t);
  o.params[0] = p;
  return one_op(q, o);
}

int mixDepolarising(Qureg q, int t, double p) {
  QSOp o = blank(QS_OP_DEPOL, t);
  o.params[0] = p;
  return one_op(q, o);
}

int calcTotalProb(Qureg q, double* out) {
  return guarded([&] {
    need(out, "out");
    Reg& r = reg_of(q);
    *out = reduce_total(*r.env, r);
  });
}

int calcProbOfOutcome(Qureg q, int qubit, int outcome, double* out) {
  return guarded([&] {
    need(out, "out");
    Reg& r = reg_of(q);
    check_qubit(r, qubit, "measured");
    if (outcome != 0 && outcome != 1) fail(QS_E_PROB, "outcome must be 0 or 1");
    *out = reduce_outcome(*r.env, r, qubit, outcome);
  });
}

int collapseToOutcome(Qureg q, int qubit, int outcome, double* probOut) {
  return guarded([&] {
    Reg& r = reg_of(q);
    check_qubit(r, qubit, "measured");
    if (outcome != 0 && outcome != 1) fail(QS_E_PROB, "outcome must be 0 or 1");
    const double p = reduce_outcome(*r.env, r, qubit, outcome);
    const double pmin = r.prec == QS_C128 ? 1e-13 : 1e-6;
    if (!(p >= pmin))
      fail(QS_E_ZERO_PROB, "outcome probability " + std::to_string(p) + " below " + std::to_string(pmin));
    launch_collapse(*r.env, r, qubit, outcome, r.density ? 1.0 / p : 1.0 / std::sqrt(p));
    if (probOut) *probOut = p;
  });
}

int calcPurity(Qureg q, double* out) {
  return guarded([&] {
    need(out, "out");
    Reg& r = reg_of(q);
    if (!r.density) fail(QS_E_NOT_DENSITY, "purity of a state vector");
    *out = reduce_purity(*r.env, r);
  });
}

int calcInnerProduct(Qureg bra, Qureg ket, Complex* out) {
  return guarded([&] {
    need(out, "out");
    Reg& a = reg_of(bra);
    Reg& b = reg_of(ket);
    if (a.density || b.density) fail(QS_E_NOT_DENSITY, "inner product of state vectors only");
    if (a.n != b.n) fail(QS_E_QUBIT, "registers of different sizes");
    const std::complex<double> z = reduce_inner(*a.env, a, b);
    out->re = z.real();
    out->im = z.imag();
  });
}

int calcFidelity(Qureg a, Qureg b, double* out) {
  return guarded([&] {
    need(out, "out");
    Reg& ra = reg_of(a);
    Reg& rb = reg_of(b);
    if (ra.density || rb.density) fail(QS_E_NOT_DENSITY, "fidelity of state vectors only");
    if (ra.n != rb.n) fail(QS_E_QUBIT, "registers of different sizes");
    *out = std::norm(reduce_inner(*ra.env, ra, rb));
  });
}

int getKernelStats(QuESTEnv e, QSKernelStat* out, int maxOut, int* count) {
  return guarded([&] {
    Env& env = env_of(e);
    need(count, "count");
    if (maxOut > 0) need(out, "out");
    QS_CUDA(cudaStreamSynchronize(env.stream));
    env.prof.collect();
    *count = int(env.prof.stats.size());
    for (int i = 0; i < maxOut && i < *count; ++i) {
      const KStat& k = env.prof.stats[i];
      std::memset(&out[i], 0, sizeof(QSKernelStat));
      std::strncpy(out[i].name, k.name.c_str(), sizeof(out[i].name) - 1);
      out[i].launches = k.launches;
      out[i].total_ms = k.ms;
      out[i].bytes = k.bytes;
      out[i].flops = k.flops;
      out[i].alu_ops = k.alu;
    }
  });
}

int resetKernelStats(QuESTEnv e) {
  return guarded([&] {
    Env& env = env_of(e);
    QS_CUDA(cudaStreamSynchronize(env.stream));
    env.prof.reset();
  });
}

int applyCircuit(Qureg q, const QSOp* ops, int64_t n) {
  return guarded([&] {
    Reg& r = reg_of(q);
    if (n < 0) fail(QS_E_ARG, "numOps < 0");
    if (n > 0) need(ops, "ops");
    std::vector<GateOp> conv;
    conv.reserve(size_t(n));
    for (int64_t i = 0; i < n; ++i) {
      try {
        convert_op(r, ops[i], conv);
      } catch (Error& e) {
        e.msg = "op " + std::to_string(i) + ": " + e.msg;
        throw;
      }
    }
    for (auto& op : conv) apply(r, op);
  });
}

}  // extern "C"
