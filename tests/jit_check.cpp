// Host-side check of the runtime-compiled pass kernels (test
// infrastructure; built by tests/test_jit.py with the host compiler against
// the library's planner, op validation and kernel generator, no GPU
// involved).
//
// Reads QSOp records from stdin, plans them for a register of the given
// shape, generates the pass kernel of every pass and compiles it with NVRTC
// for sm_103a.  Prints "JIT passes P compiled C distinct D seconds S" and,
// for a failure, the compiler log.  copy = 1 / 2 generates the bulk-copy /
// async-copy pipeline form.  Argument 8 caps how many distinct kernels are compiled
// (all are generated); with a file name as argument 9 the source of the
// first pass is written there.  Compiles run on up to 8
// host threads.
//
// usage: jit_check n density prec arith k_req ctas copy [max_compile [source_out]]
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "jit.h"
#include "jit_runtime.h"
#include "plan.h"
#include "runtime.h"

using namespace qs;

// jit.cpp's launch path (never called here) times launches with KTimer,
// which lives in the CUDA part of the library
namespace qs {
KTimer::KTimer(Env& env, const char*, double, double, int, double) : env_(env) {}
KTimer::~KTimer() {}
}  // namespace qs

int main(int argc, char** argv) {
  if (argc < 8) {
    std::fprintf(stderr, "usage: jit_check n density prec arith k_req ctas copy [max_compile [source_out]]\n");
    return 2;
  }
  const int n = std::atoi(argv[1]), density = std::atoi(argv[2]), prec = std::atoi(argv[3]);
  const int arith = std::atoi(argv[4]), k_req = std::atoi(argv[5]), ctas = std::atoi(argv[6]);
  const int copy = std::atoi(argv[7]);
  Env env;
  env.arith = arith;
  // the "tile_low_qubits" option (contiguous low qubits per tile), if set
  if (const char* t = std::getenv("JIT_CHECK_TILE_LOW")) env.tile_low_qubits = std::atoi(t);
  Reg r;
  r.env = &env;
  r.n = n;
  r.density = density != 0;
  r.nq = density ? 2 * n : n;
  r.prec = prec;
  r.dim = int64_t(1) << r.nq;
  std::vector<QSOp> ops;
  QSOp o;
  while (std::fread(&o, sizeof(o), 1, stdin) == 1) ops.push_back(o);
  RegPlan pl;
  try {
    std::vector<GateOp> g;
    convert_ops(r, ops.data(), int64_t(ops.size()), g);
    build_plan(r, g, k_req, (uint64_t(1) << r.nq) - 1, 1.0, pl);
  } catch (const Error& e) {
    std::printf("ERROR %d %s\n", e.code, e.msg.c_str());
    return 1;
  }
  const int R = pl.arith == Arith::F32 ? 5 : 4;
  const int max_compile = argc > 8 ? std::atoi(argv[8]) : 1 << 30;
  JitShape shape{pl.arith, R, ctas};
  shape.copy = static_cast<JitCopy>(copy % 4);
  shape.direct_store = (copy & 4) != 0;  // copy + 4: the last stage stores to HBM
  shape.swizzle = (copy & 8) == 0;       // copy + 8: no shared-memory swizzle
  std::set<std::string> distinct;
  std::vector<std::string> todo;
  for (size_t i = 0; i < pl.fps.size(); ++i) {
    std::string src;
    try {
      src = jit_source(pl.fps[i], pl.fst.data(), pl.fops.data(), shape);
    } catch (const Error& e) {
      std::printf("GENFAIL pass %zu: %s\n", i, e.msg.c_str());
      return 3;
    }
    if (argc > 9 && (i == 0 || std::getenv("JIT_CHECK_ALL"))) {
      const std::string name = std::string(argv[9]) + (i == 0 ? "" : "." + std::to_string(i));
      FILE* f = std::fopen(name.c_str(), "w");
      if (f) {
        std::fputs(src.c_str(), f);
        std::fclose(f);
      }
    }
    if (distinct.insert(src).second && int(todo.size()) < max_compile) todo.push_back(src);
  }
  std::vector<int> ok(todo.size(), 0);
  std::vector<std::string> logs(todo.size());
  std::vector<std::thread> th;
  const auto t0 = std::chrono::steady_clock::now();
  const size_t nth = std::min<size_t>(8, todo.size());
  for (size_t w = 0; w < nth; ++w)
    th.emplace_back([&, w] {
      for (size_t i = w; i < todo.size(); i += nth) {
        std::vector<char> cubin;
        ok[i] = jit_compile_cubin(todo[i], cubin, logs[i]) ? 1 : 0;
      }
    });
  for (std::thread& t : th) t.join();
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int compiled = 0;
  for (size_t i = 0; i < todo.size(); ++i) {
    if (!ok[i]) {
      std::printf("COMPILEFAIL kernel %zu\n%s\n", i, logs[i].c_str());
      return 4;
    }
    ++compiled;
  }
  std::printf("JIT passes %zu compiled %d distinct %zu seconds %.3f\n", pl.fps.size(), compiled, distinct.size(),
              secs);
  return 0;
}
