// Serving loop: requests (one circuit each) admitted onto the GPU as slots
// and memory free up.
//
// serveCreate starts a scheduler thread and `slots` execution slots.  Each
// slot owns a private environment (its own CUDA stream and reduction
// scratch) whose registers are allocated stream-ordered (cudaMallocAsync /
// cudaFreeAsync on the slot's stream), so admitting or retiring a request
// never synchronises the device.  serveSubmit validates a request and
// queues it.  The scheduler admits queued requests in arrival order while a
// slot is free and the register fits the memory budget, queues the
// register's |0...0>, its fused circuit, the FP64 reductions and the result
// copy on the slot's stream, and learns of completion from a host function
// queued behind them (cudaLaunchHostFunc), so requests on different slots
// run concurrently on the device and no kernel ever waits for another.
// servePoll waits, with a caller-given limit, for one request's result.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "runtime.h"

namespace qs {

namespace {

using Clock = std::chrono::steady_clock;

double us_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::micro>(b - a).count();
}

struct Server;

struct Request {
  int64_t ticket = 0;
  QSRequest req{};
  std::vector<QSOp> ops;
  int64_t bytes = 0;
  Clock::time_point submit, admit;
  QSResult result{};
  bool finished = false;
};

struct Slot {
  Server* srv = nullptr;
  int index = 0;
  QuESTEnv env{0};
  Env* e = nullptr;
  Request* cur = nullptr;
  Qureg q{0};
  std::atomic<bool> gpu_done{false};
  Clock::time_point t_done;
};

struct Server {
  int64_t id = 0;
  int device = 0;
  int64_t budget = 0, used = 0;
  std::vector<Slot*> slots;
  std::deque<Request*> queue;
  std::unordered_map<int64_t, Request*> tickets;
  std::mutex mu;
  std::condition_variable cv;       // wakes the scheduler
  std::condition_variable done_cv;  // wakes pollers
  bool stop = false;
  std::thread th;
  int64_t next_ticket = 1;
  // admission policy (0 = none): queue length past which serveSubmit
  // refuses, queue wait after which a request is shed
  int64_t max_queue = 0, max_queue_us = 0;
  int64_t shed = 0, refused = 0;
  // the device's default pool: its release threshold before the server
  // raised it (restored, and the cached blocks released, when it stops)
  cudaMemPool_t pool = nullptr;
  uint64_t pool_threshold = 0;
};

std::mutex g_smu;
std::unordered_map<int64_t, Server*> g_servers;
int64_t g_next_server = 1;

void* slot_alloc(size_t bytes, void* ctx) {
  Slot* s = static_cast<Slot*>(ctx);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s->e->stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void slot_release(void* p, void* ctx) {
  Slot* s = static_cast<Slot*>(ctx);
  cudaFreeAsync(p, s->e->stream);
}

// Runs on a CUDA-owned thread once the slot's queued work has finished: no
// CUDA calls here, only the flag, the time and a wake-up.
void CUDART_CB on_slot_done(void* p) {
  Slot* s = static_cast<Slot*>(p);
  s->t_done = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->srv->mu);
    s->gpu_done.store(true);
  }
  s->srv->cv.notify_one();
}

// Queues one request's work on a free slot (scheduler thread, no lock held).
int start(Slot& s, Request& r) {
  const QSRequest& q = r.req;
  int st = q.isDensity ? createDensityQureg(q.numQubits, q.precision, s.env, &s.q)
                       : createQureg(q.numQubits, q.precision, s.env, &s.q);
  if (st != QS_OK) return st;
  st = applyCircuit(s.q, r.ops.data(), int64_t(r.ops.size()));
  if (st != QS_OK) return st;
  return guarded_call([&] {
    Reg& reg = lookup_reg(s.q.id);
    Env& e = *s.e;
    queue_total(e, reg, e.d_result);
    queue_outcome(e, reg, q.measureQubit, 0, e.d_result + 1);
    QS_CUDA(cudaMemcpyAsync(e.h_result, e.d_result, 2 * sizeof(double), cudaMemcpyDeviceToHost, e.stream));
    s.gpu_done.store(false);
    QS_CUDA(cudaLaunchHostFunc(e.stream, on_slot_done, &s));
  });
}

// Collects a finished slot's results and frees its register (scheduler
// thread, no lock held).  Returns the request's status.
int finish(Slot& s, Request& r) {
  r.result.totalProb = s.e->h_result[0];
  r.result.probOutcome0 = s.e->h_result[1];
  int st = QS_OK;
  if (r.req.outAmps && r.req.outCount > 0) st = copyStateToHost(s.q, r.req.outAmps, 0, r.req.outCount);
  destroyQureg(s.q);
  s.q.id = 0;
  return st;
}

void scheduler(Server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    // completions
    for (Slot* s : S->slots) {
      if (!s->cur || !s->gpu_done.load()) continue;
      Request* r = s->cur;
      lk.unlock();
      const int st = finish(*s, *r);
      lk.lock();
      r->result.status = st;
      r->result.latencyUs = us_between(r->submit, s->t_done);
      r->finished = true;
      S->used -= r->bytes;
      s->cur = nullptr;
      s->gpu_done.store(false);
      S->done_cv.notify_all();
    }
    // shedding: requests that waited longer than the bound leave the queue
    // with QS_E_BUSY (admitted requests then never wait longer)
    if (S->max_queue_us > 0 && !S->queue.empty()) {
      const Clock::time_point now = Clock::now();
      for (auto it = S->queue.begin(); it != S->queue.end();) {
        Request* r = *it;
        if (us_between(r->submit, now) > double(S->max_queue_us)) {
          r->result.status = QS_E_BUSY;
          r->result.slot = -1;
          r->result.queuedUs = us_between(r->submit, now);
          r->result.latencyUs = r->result.queuedUs;
          r->finished = true;
          ++S->shed;
          it = S->queue.erase(it);
        } else {
          ++it;
        }
      }
      S->done_cv.notify_all();
    }
    // admissions: arrival order, while a slot is free and the budget allows
    while (!S->stop && !S->queue.empty()) {
      Request* r = S->queue.front();
      if (S->used + r->bytes > S->budget) break;
      Slot* free_slot = nullptr;
      for (Slot* s : S->slots)
        if (!s->cur) {
          free_slot = s;
          break;
        }
      if (!free_slot) break;
      S->queue.pop_front();
      S->used += r->bytes;
      free_slot->cur = r;
      r->admit = Clock::now();
      r->result.slot = free_slot->index;
      r->result.queuedUs = us_between(r->submit, r->admit);
      lk.unlock();
      const int st = start(*free_slot, *r);
      lk.lock();
      if (st != QS_OK) {  // could not be queued: report and free the slot
        lk.unlock();
        cudaStreamSynchronize(free_slot->e->stream);
        if (free_slot->q.id) destroyQureg(free_slot->q);
        lk.lock();
        free_slot->q.id = 0;
        free_slot->cur = nullptr;
        S->used -= r->bytes;
        r->result.status = st;
        r->result.latencyUs = us_between(r->submit, Clock::now());
        r->finished = true;
        S->done_cv.notify_all();
      }
    }
    bool busy = false;
    for (Slot* s : S->slots) busy = busy || s->cur;
    if (S->stop && !busy) break;
    S->cv.wait_for(lk, std::chrono::milliseconds(50), [&] {
      if (S->stop) return true;
      for (Slot* s : S->slots)
        if (s->cur && s->gpu_done.load()) return true;
      if (S->queue.empty()) return false;
      bool free_slot = false;
      for (Slot* s : S->slots) free_slot = free_slot || !s->cur;
      return free_slot && S->used + S->queue.front()->bytes <= S->budget;
    });
  }
  // cancelled requests still queued at shutdown
  for (Request* r : S->queue) {
    r->result.status = QS_E_ARG;
    r->finished = true;
  }
  S->queue.clear();
  S->done_cv.notify_all();
}

Server& server_of(QSServer h) {
  std::lock_guard<std::mutex> lk(g_smu);
  auto it = g_servers.find(h.id);
  if (it == g_servers.end()) fail(QS_E_HANDLE, "unknown server handle " + std::to_string(h.id));
  return *it->second;
}

}  // namespace

}  // namespace qs

using namespace qs;

extern "C" {

int serveCreate(QuESTEnv env, int slots, int64_t budgetBytes, int fusion, QSServer* out) {
  return guarded_call([&] {
    if (!out) fail(QS_E_ARG, "null output");
    if (slots < 1 || slots > 64) fail(QS_E_ARG, "slots must be in 1..64");
    if (budgetBytes < 1) fail(QS_E_ARG, "budget must be positive");
    if (fusion != 0 && fusion != 1) fail(QS_E_ARG, "fusion must be 0 or 1");
    Env& parent = lookup_env(env.id);
    auto* S = new Server();
    S->device = parent.device;
    S->budget = budgetBytes;
    try {
      QS_CUDA(cudaSetDevice(S->device));
      cudaMemPool_t pool;
      QS_CUDA(cudaDeviceGetDefaultMemPool(&pool, S->device));
      QS_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &S->pool_threshold));
      S->pool = pool;
      uint64_t keep = ~uint64_t(0);  // keep freed blocks cached in the pool while serving
      QS_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
      for (int i = 0; i < slots; ++i) {
        auto* s = new Slot();
        s->srv = S;
        s->index = i;
        S->slots.push_back(s);
        int st = createQuESTEnv(&s->env);
        if (st != QS_OK) fail(st, qsLastError());
        s->e = &lookup_env(s->env.id);
        s->e->fusion = fusion;
        s->e->arith = parent.arith;
        s->e->tile_qubits = parent.tile_qubits;
        st = setAllocator(s->env, slot_alloc, slot_release, s);
        if (st != QS_OK) fail(st, qsLastError());
      }
    } catch (...) {
      for (Slot* s : S->slots) {
        if (s->env.id) destroyQuESTEnv(s->env);
        delete s;
      }
      delete S;
      throw;
    }
    S->th = std::thread(scheduler, S);
    std::lock_guard<std::mutex> lk(g_smu);
    S->id = g_next_server++;
    g_servers[S->id] = S;
    out->id = S->id;
  });
}

int serveSubmit(QSServer h, const QSRequest* req, int64_t* ticket) {
  return guarded_call([&] {
    if (!req || !ticket) fail(QS_E_ARG, "null pointer");
    Server& S = server_of(h);
    if (req->precision != QS_C64 && req->precision != QS_C128) fail(QS_E_ARG, "bad precision");
    const int nq = req->isDensity ? 2 * req->numQubits : req->numQubits;
    if (req->numQubits < 1 || nq > 40) fail(QS_E_QUBIT, "unsupported qubit count");
    if (req->measureQubit < 0 || req->measureQubit >= req->numQubits) fail(QS_E_QUBIT, "measureQubit out of range");
    if (req->numOps < 0 || (req->numOps > 0 && !req->ops)) fail(QS_E_ARG, "bad op list");
    if (req->outAmps && (req->outCount < 0 || req->outCount > (int64_t(1) << nq)))
      fail(QS_E_ARG, "outCount out of range");
    // validate the circuit against a register of this shape (nothing allocated)
    Reg shape;
    shape.n = req->numQubits;
    shape.density = req->isDensity != 0;
    shape.nq = nq;
    shape.prec = req->precision;
    shape.dim = int64_t(1) << nq;
    std::vector<GateOp> tmp;
    convert_ops(shape, req->ops, req->numOps, tmp);
    auto* r = new Request();
    r->req = *req;
    r->ops.assign(req->ops, req->ops + req->numOps);
    r->req.ops = nullptr;
    r->bytes = shape.dim * (req->precision == QS_C128 ? 16 : 8);
    r->submit = Clock::now();
    if (r->bytes > S.budget) {
      delete r;
      fail(QS_E_NOMEM, "request larger than the server's memory budget");
    }
    {
      std::lock_guard<std::mutex> lk(S.mu);
      if (S.stop) {
        delete r;
        fail(QS_E_ARG, "server is shutting down");
      }
      if (S.max_queue > 0 && int64_t(S.queue.size()) >= S.max_queue) {
        ++S.refused;
        delete r;
        fail(QS_E_BUSY, "the server's queue is full (max_queue)");
      }
      r->ticket = S.next_ticket++;
      S.tickets[r->ticket] = r;
      S.queue.push_back(r);
      *ticket = r->ticket;
    }
    S.cv.notify_one();
  });
}

int servePoll(QSServer h, int64_t ticket, QSResult* out, int64_t timeoutUs) {
  return guarded_call([&] {
    if (!out) fail(QS_E_ARG, "null output");
    if (timeoutUs < 0) fail(QS_E_ARG, "timeout must be >= 0 microseconds");
    Server& S = server_of(h);
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.tickets.find(ticket);
    if (it == S.tickets.end()) fail(QS_E_HANDLE, "unknown or already collected ticket");
    Request* r = it->second;
    S.done_cv.wait_for(lk, std::chrono::microseconds(timeoutUs), [&] { return r->finished; });
    if (!r->finished) fail(QS_E_TIMEOUT, "request not finished within the timeout");
    *out = r->result;
    S.tickets.erase(it);
    delete r;
  });
}

int serveSetOption(QSServer h, const char* key, int64_t value) {
  return guarded_call([&] {
    if (!key) fail(QS_E_ARG, "null key");
    Server& S = server_of(h);
    const std::string k(key);
    if (value < 0) fail(QS_E_ARG, k + " must be >= 0");
    std::lock_guard<std::mutex> lk(S.mu);
    if (k == "max_queue") S.max_queue = value;
    else if (k == "max_queue_us") S.max_queue_us = value;
    else fail(QS_E_ARG, "unknown server option " + k);
    S.cv.notify_one();
  });
}

int serveGetOption(QSServer h, const char* key, int64_t* value) {
  return guarded_call([&] {
    if (!key || !value) fail(QS_E_ARG, "null pointer");
    Server& S = server_of(h);
    const std::string k(key);
    std::lock_guard<std::mutex> lk(S.mu);
    if (k == "max_queue") *value = S.max_queue;
    else if (k == "max_queue_us") *value = S.max_queue_us;
    else if (k == "queued") *value = int64_t(S.queue.size());
    else if (k == "shed") *value = S.shed;
    else if (k == "refused") *value = S.refused;
    else fail(QS_E_ARG, "unknown server option " + k);
  });
}

int serveDestroy(QSServer h) {
  return guarded_call([&] {
    Server* S = &server_of(h);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
    }
    S->cv.notify_all();
    S->th.join();
    for (Slot* s : S->slots) {
      destroyQuESTEnv(s->env);
      delete s;
    }
    for (auto& kv : S->tickets) delete kv.second;
    // give the pool's cached blocks back and restore its threshold: the
    // server's setting must not outlive it
    if (S->pool) {
      cudaDeviceSynchronize();
      cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &S->pool_threshold);
      cudaMemPoolTrimTo(S->pool, 0);
    }
    {
      std::lock_guard<std::mutex> lk(g_smu);
      g_servers.erase(S->id);
    }
    delete S;
  });
}

}  // extern "C"
