// Per-kernel-class event timing.
#include "runtime.h"

namespace qs {

int Profiler::class_of(const std::string& name) {
  for (size_t i = 0; i < stats.size(); ++i)
    if (stats[i].name == name) return int(i);
  stats.push_back(KStat{name});
  return int(stats.size() - 1);
}

cudaEvent_t Profiler::event() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  QS_CUDA(cudaEventCreate(&e));
  return e;
}

void Profiler::collect() {
  for (const KPending& p : pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) stats[p.cls].ms += ms;
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
}

void Profiler::reset() {
  collect();
  stats.clear();
}

KTimer::KTimer(Env& env, const char* name, double bytes, double flops, int nlaunch, double alu)
    : env_(env) {
  env.launches += nlaunch;
  if (!env.profile) return;
  cls_ = env.prof.class_of(name);
  KStat& s = env.prof.stats[cls_];
  s.launches += 1;
  s.bytes += bytes;
  s.flops += flops;
  s.alu += alu;
  a_ = env.prof.event();
  cudaEventRecord(a_, env.stream);
}

KTimer::~KTimer() {
  if (cls_ < 0) return;
  cudaEvent_t b = env_.prof.event();
  cudaEventRecord(b, env_.stream);
  env_.prof.pending.push_back(KPending{cls_, a_, b});
}

}  // namespace qs
