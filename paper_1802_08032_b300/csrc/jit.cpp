// Runtime compilation and cache of the generated pass kernels (see jit.h).
//
// A kernel is compiled by NVRTC for sm_103a straight to a cubin, loaded as
// a context-independent CUDA library and kept for the life of the process,
// keyed by its source text (which spells out the whole pass structure, so
// equal text means an equal kernel).  Compilation runs on a small pool of
// host threads: with the "jit" option 2 (asynchronous) a flush launches the
// interpreting kernel for any pass whose kernel is not ready yet and queues
// its compilation; with 1 (synchronous) the flush waits for the compile.
// The compile threads make no CUDA calls: a compiled cubin is loaded by the
// next flush that needs it, on the caller's thread, so nothing in the
// background touches the CUDA runtime (a compile still running when the
// process exits is waited for and discarded).
#include <nvrtc.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "jit.h"
#include "jit_runtime.h"
#include "runtime.h"

namespace qs {

// Headers embedded at build time (generated jit_headers.inc: an array of
// {name, text} pairs of the device headers the generated source includes).
namespace {
struct EmbeddedHeader {
  const char* name;
  const char* text;
};
#include "jit_headers.inc"
}  // namespace

int jit_header_count() { return int(sizeof(kJitHeaders) / sizeof(kJitHeaders[0])); }
const char* jit_header_name(int i) { return kJitHeaders[i].name; }
const char* jit_header_text(int i) { return kJitHeaders[i].text; }

namespace {

// SEEN (met once, not compiled) -> QUEUED -> COMPILED (cubin ready, by a
// compile thread) -> READY (loaded, by a caller's thread); or FAILED.
enum JitState : int { JS_QUEUED = 0, JS_READY = 1, JS_FAILED = 2, JS_COMPILED = 3, JS_SEEN = 4 };

struct JitEntry {
  std::string src;
  size_t smem = 0;
  std::atomic<int> state{JS_QUEUED};
  std::vector<char> cubin;
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kern = nullptr;
  double compile_s = 0;
  std::string log;
};

class JitCache {
 public:
  static JitCache& get() {
    static JitCache c;
    return c;
  }
  ~JitCache() { shutdown(); }

  // Drops queued compiles, waits for the ones in flight and ends the
  // compile threads (they start again on the next queued compile).  Must
  // run before the process exits: NVRTC's own static data may be torn down
  // before this object's destructor, under a compile still running.
  void shutdown() {
    std::vector<std::thread> ws;
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
      for (auto& e : queue_) e->state.store(JS_SEEN);  // not compiled: met again, queued again
      queue_.clear();
      ws.swap(workers_);
    }
    cv_.notify_all();
    for (std::thread& t : ws)
      if (t.joinable()) t.join();
    std::lock_guard<std::mutex> lk(mu_);
    stop_ = false;
    done_cv_.notify_all();
  }

  // The entry of this source.  A structure is queued for compilation the
  // second time it is met (or at once with now = true): circuits that are
  // never rerun (serving, one-off circuits) cost no compile.  At most
  // kSeenMax structures met only once are remembered (oldest forgotten).
  std::shared_ptr<JitEntry> find_or_queue(const std::string& src, size_t smem, bool now) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = map_.find(src);
    std::shared_ptr<JitEntry> e;
    if (it != map_.end()) {
      e = it->second;
      if (e->state.load() != JS_SEEN) return e;
    } else {
      e = std::make_shared<JitEntry>();
      e->src = src;
      e->smem = smem;
      e->state.store(JS_SEEN);
      map_.emplace(src, e);
      seen_.push_back(src);
      if (seen_.size() > kSeenMax) {
        auto old = map_.find(seen_.front());
        if (old != map_.end() && old->second->state.load() == JS_SEEN) map_.erase(old);
        seen_.pop_front();
      }
      if (!now) return e;
    }
    e->state.store(JS_QUEUED);
    queue_.push_back(e);
    start_workers_locked();
    cv_.notify_one();
    return e;
  }

  // Waits until e is compiled (or failed).
  void wait(const std::shared_ptr<JitEntry>& e) {
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return e->state.load() != JS_QUEUED || stop_; });
  }

  // Loads a compiled cubin (caller's thread, the device current); true
  // when e is ready to launch.
  bool load(JitEntry& e) {
    std::lock_guard<std::mutex> lk(load_mu_);
    if (e.state.load() == JS_READY) return true;
    if (e.state.load() != JS_COMPILED) return false;
    cudaError_t err = cudaLibraryLoadData(&e.lib, e.cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (err == cudaSuccess) err = cudaLibraryGetKernel(&e.kern, e.lib, "qs_pass");
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(reinterpret_cast<const void*>(e.kern), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(e.smem));
    if (err != cudaSuccess) {
      cudaGetLastError();
      e.log = std::string("load: ") + cudaGetErrorString(err);
      e.state.store(JS_FAILED);
      return false;
    }
    e.cubin.clear();
    e.cubin.shrink_to_fit();
    e.state.store(JS_READY);
    return true;
  }

  JitStats stats() {
    std::lock_guard<std::mutex> lk(mu_);
    JitStats s{};
    for (auto& kv : map_) {
      const int st = kv.second->state.load();
      if (st == JS_READY || st == JS_COMPILED) {
        ++s.ready;
        s.compile_s += kv.second->compile_s;
      } else if (st == JS_FAILED) {
        ++s.failed;
      } else if (st == JS_QUEUED) {
        ++s.pending;
      }
    }
    return s;
  }

  std::string first_failure() {
    std::lock_guard<std::mutex> lk(mu_);
    for (auto& kv : map_)
      if (kv.second->state.load() == JS_FAILED) return kv.second->log;
    return {};
  }

 private:
  void start_workers_locked() {
    if (!workers_.empty()) return;
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const unsigned n = std::min(16u, std::max(2u, hw / 2));
    for (unsigned i = 0; i < n; ++i) workers_.emplace_back([this] { run(); });
  }

  void run() {
    for (;;) {
      std::shared_ptr<JitEntry> e;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || !queue_.empty(); });
        if (stop_) return;
        e = queue_.front();
        queue_.pop_front();
      }
      compile(*e);
      {
        std::lock_guard<std::mutex> lk(mu_);  // (orders the state change before waiters check it)
      }
      done_cv_.notify_all();
    }
  }

  // NVRTC only: no CUDA runtime call on a compile thread.
  static void compile(JitEntry& e) {
    const auto t0 = std::chrono::steady_clock::now();
    std::string log;
    std::vector<char> cubin;
    const bool ok = jit_compile_cubin(e.src, cubin, log);
    if (ok) {
      e.cubin = std::move(cubin);
      e.compile_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      e.state.store(JS_COMPILED);
    } else {
      e.log = log;
      e.state.store(JS_FAILED);
    }
  }

  std::mutex mu_, load_mu_;
  std::condition_variable cv_, done_cv_;
  bool stop_ = false;
  std::deque<std::shared_ptr<JitEntry>> queue_;
  std::deque<std::string> seen_;  // structures met once, oldest first
  static constexpr size_t kSeenMax = 1024;
  std::unordered_map<std::string, std::shared_ptr<JitEntry>> map_;
  std::vector<std::thread> workers_;
};

}  // namespace

bool jit_compile_cubin(const std::string& src, std::vector<char>& cubin, std::string& log) {
  const int nh = jit_header_count();
  std::vector<const char*> hdr(static_cast<size_t>(nh)), names(static_cast<size_t>(nh));
  for (int i = 0; i < nh; ++i) {
    hdr[size_t(i)] = jit_header_text(i);
    names[size_t(i)] = jit_header_name(i);
  }
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "qs_pass.cu", nh, hdr.data(), names.data()) != NVRTC_SUCCESS) {
    log = "nvrtcCreateProgram failed";
    return false;
  }
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device", "-lineinfo"};
  const nvrtcResult r = nvrtcCompileProgram(prog, 4, opts);
  size_t ls = 0;
  nvrtcGetProgramLogSize(prog, &ls);
  if (ls > 1) {
    log.resize(ls);
    nvrtcGetProgramLog(prog, &log[0]);
  }
  bool ok = r == NVRTC_SUCCESS;
  if (ok) {
    size_t cs = 0;
    ok = nvrtcGetCUBINSize(prog, &cs) == NVRTC_SUCCESS && cs > 0;
    if (ok) {
      cubin.resize(cs);
      ok = nvrtcGetCUBIN(prog, cubin.data()) == NVRTC_SUCCESS;
    }
  } else {
    log = std::string(nvrtcGetErrorString(r)) + ": " + log;
  }
  nvrtcDestroyProgram(&prog);
  return ok;
}

bool jit_try_launch(Env& env, Reg& r, const FPass& fp, const FStage* st, const FOp* ops, Arith arith, int R,
                    double flops, double alu, const char* name, RegPlan::JitMemo* memo, size_t pass_index) {
  if (!jit_wanted(env, r, arith) || fp.init) return false;
  if (fp.op_count <= 0 || fp.op_count > kMaxPassOps) return false;
  const JitCopy copy = jit_copy_mode(env, arith);
  JitShape sh{arith, R, jit_ctas_for(env, fp, arith, copy)};
  sh.copy = copy;
  sh.direct_store = env.jit_direct != 0;
  sh.swizzle = env.jit_swizzle != 0;
  const size_t smem = jit_smem_bytes(fp, sh);
  // a plan met before with this kernel shape: its entry, without
  // generating the source again
  const uint64_t sig = (uint64_t(arith) << 0) | (uint64_t(R) << 4) | (uint64_t(sh.ctas) << 8) |
                       (uint64_t(int(copy)) << 12) | (uint64_t(sh.direct_store) << 16) |
                       (uint64_t(sh.swizzle) << 17) | (uint64_t(1) << 20);
  std::shared_ptr<JitEntry> e;
  if (memo) {
    if (memo->sig != sig) {
      memo->sig = sig;
      memo->kernels.clear();
    }
    if (memo->kernels.size() <= pass_index) memo->kernels.resize(pass_index + 1);
    e = std::static_pointer_cast<JitEntry>(memo->kernels[pass_index]);
    if (e && e->state.load() == JS_SEEN) e = nullptr;  // met once: look it up (and queue it) again
  }
  if (!e) {
    std::string src;
    try {
      src = jit_source(fp, st, ops, sh);
    } catch (const Error&) {
      ++env.jit_rejected;
      return false;
    }
    e = JitCache::get().find_or_queue(src, smem, env.jit == 1);
    if (memo) memo->kernels[pass_index] = e;
  }
  if (env.jit == 1 && e->state.load() == JS_QUEUED) JitCache::get().wait(e);
  if (!JitCache::get().load(*e)) return false;
  // parameters: g, ntiles, then the pass's FOp records (constant bank)
  void* g = r.d;
  long long ntiles = fp.ntiles;
  unsigned* status = env.d_status;
  const FOp* popv = ops + fp.op_begin;
  void* args_plain[3] = {&g, &ntiles, const_cast<FOp*>(popv)};
  void* args_bulk[4] = {&g, &ntiles, &status, const_cast<FOp*>(popv)};
  void** args = sh.copy == JitCopy::Bulk ? args_bulk : args_plain;
  const int threads = 1 << (fp.k - R);
  const int64_t grid = std::min<int64_t>(fp.ntiles, int64_t(env.sms) * sh.ctas);
  const double bytes = std::ldexp(2.0 * (arith == Arith::F32 ? 8.0 : 16.0), r.nq);
  KTimer kt(env, name, bytes, flops, 1, alu);
  QS_CUDA(cudaLaunchKernel(reinterpret_cast<const void*>(e->kern), dim3(unsigned(grid)), dim3(unsigned(threads)),
                           args, smem, env.stream));
  ++env.jit_launches;
  return true;
}

JitStats jit_stats() { return JitCache::get().stats(); }
void jit_shutdown() { JitCache::get().shutdown(); }
std::string jit_first_failure() { return JitCache::get().first_failure(); }

}  // namespace qs
