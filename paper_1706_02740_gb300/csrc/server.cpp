// Serving loop (sft_server_*): admission by device-memory budget, resident plans and continuous
// batching over several streams.
//
// Threads: callers submit and query under one mutex; one scheduler thread owns the plans, the
// arena and the launch slots; builder threads (sft_server_config.build_threads) build the plans
// of requests whose (N, s) has no idle resident plan, so a new N does not hold up the requests
// queued behind it (they are batched while it builds, and it joins the next batch once its plan
// is ready); CUDA's host-callback thread marks a slot done when its batched execution has
// finished on the device.  The scheduler makes no CUDA call while it holds the mutex, so a
// completion callback never waits on CUDA work.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "arena.h"
#include "alloc_hook.h"
#include "guard.h"
#include "sft_internal.h"

namespace sft {
namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int kMaxServerBatch = 256;
constexpr int kMaxInflight = 8;
constexpr int kMaxBuilders = 16;

// The budget as device memory: one cudaMalloc, blocks handed out by OffsetArena, uploads on a
// private non-blocking stream (never the legacy default stream, which would wait for other work).
class DeviceArena final : public DeviceMemory {
 public:
  ~DeviceArena() override {
    if (st_) cudaStreamDestroy(st_);
    if (base_) cudaFree(base_);
  }
  cudaError_t init(size_t bytes) {
    book_.reset(bytes);
    cudaError_t e = dev_malloc((void**)&base_, book_.capacity());
    if (e != cudaSuccess) {
      base_ = nullptr;
      return e;
    }
    return cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking);
  }
  void* alloc(size_t bytes) override {
    std::lock_guard<std::mutex> g(mu_);
    const int64_t off = book_.alloc(bytes);
    return off < 0 ? nullptr : base_ + off;
  }
  void release(void* p) override {
    std::lock_guard<std::mutex> g(mu_);
    book_.release((size_t)(static_cast<char*>(p) - base_));
  }
  cudaError_t upload(void* dst, const void* src, size_t bytes) override {
    std::lock_guard<std::mutex> g(up_mu_);
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st_);
    return e == cudaSuccess ? cudaStreamSynchronize(st_) : e;
  }
  size_t largest_free() { std::lock_guard<std::mutex> g(mu_); return book_.largest_free(); }
  void usage(size_t* cap, size_t* used, size_t* peak) {
    std::lock_guard<std::mutex> g(mu_);
    *cap = book_.capacity();
    *used = book_.used();
    *peak = book_.peak();
  }

 private:
  char* base_ = nullptr;
  cudaStream_t st_ = nullptr;
  OffsetArena book_;
  std::mutex mu_, up_mu_;
};

struct Entry {                       // a resident plan
  Plan P;
  int64_t N = 0;
  int32_t s = 0;
  bool busy = false;
  std::list<Entry*>::iterator lru_it;  // position in the idle list while idle
};

struct Request {
  int64_t N = 0;
  int32_t s = 0;
  const void* f = nullptr;
  int64_t* w = nullptr;
  void* c = nullptr;
  int32_t* n = nullptr;
  int32_t state = 0;                 // 0 queued, 1 running, 2 done, 3 failed
  int32_t status = SFT_OK;
  int32_t batch_size = 0, reused = 0;
  Clock::time_point t_submit, t_launch, t_done;
  Entry* plan = nullptr;             // set when a builder made its plan (or at admission)
  double build_ms = 0.0;             // host time spent building its plan (0 when reused)
  bool build_here = false;           // a builder ran out of arena: build with eviction inline
};

struct Built {                       // a builder's result, handed to the scheduler
  int64_t id;
  Entry* e;                          // nullptr on failure
  sft_status status;
  double ms;
};

struct Server;

struct Slot {                        // one batched execution in flight
  Server* srv = nullptr;
  cudaStream_t st = nullptr;
  char* dev = nullptr;               // plan records | block prefixes | pointer arrays
  char* host = nullptr;              // pinned staging of the same
  size_t bytes = 0;
  bool busy = false;
  bool done = false;                 // set by the completion callback (under the server mutex)
  bool dead = false;                 // its stream failed: never used again
  Clock::time_point t_done;
  std::vector<int64_t> reqs;
  std::vector<Entry*> plans;
};

struct Server {
  sft_server_config cfg;
  DeviceArena arena;
  std::vector<Slot*> slots;
  std::mutex mu;
  std::condition_variable cv;        // wakes the scheduler
  std::condition_variable done_cv;   // wakes waiters
  std::thread th;
  bool stop = false;
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, Request> reqs;
  int64_t next_id = 1;
  // scheduler-thread state
  std::multimap<std::pair<int64_t, int32_t>, Entry*> plans;
  std::list<Entry*> lru;             // idle plans, least recently used first
  sft_server_stats stats;            // guarded by mu
  int device = 0;
  // plan builders (guarded by mu)
  std::vector<std::thread> builders;
  std::condition_variable build_cv;
  std::deque<int64_t> build_q;
  std::vector<Built> built;
  int building = 0;
  bool stop_builders = false;
  // shutdown: sft_server_destroy waits for the scheduler; past its limit it sets `abort`, and the
  // scheduler fails what is queued instead of running it
  bool abort = false;
  bool exited = false;
  std::condition_variable exit_cv;
};

// Builder thread: takes a request id, builds its plan from the arena (thread-safe) with the
// server's variant, and hands the plan (or the failure) back to the scheduler.
void builder(Server* Sp) {
  Server& S = *Sp;
  cudaSetDevice(S.device);
  std::unique_lock<std::mutex> lk(S.mu);
  for (;;) {
    S.build_cv.wait(lk, [&] { return S.stop_builders || !S.build_q.empty(); });
    if (S.build_q.empty()) break;
    const int64_t id = S.build_q.front();
    S.build_q.pop_front();
    const Request& r = S.reqs[id];
    const int64_t N = r.N;
    const int32_t s = r.s;
    ++S.building;
    lk.unlock();
    const auto t0 = Clock::now();
    Entry* e = new (std::nothrow) Entry();
    sft_status st = SFT_ENOMEM;
    if (e) {
      st = build_plan(&e->P, N, s, &S.cfg.variant, 0, nullptr, 0, nullptr, 0, &S.arena);
      if (st == SFT_OK) {
        e->N = N;
        e->s = s;
        e->busy = true;
      } else {
        free_plan(&e->P);
        delete e;
        e = nullptr;
      }
    }
    const double ms = ms_between(t0, Clock::now());
    lk.lock();
    --S.building;
    S.built.push_back({id, e, st, ms});
    S.cv.notify_all();
  }
}

// Hand the builders' results to the queue (scheduler thread, mu held): a built plan becomes
// resident (busy, for its request) and its request goes to the front of the queue; a request
// whose build ran out of arena is retried by the scheduler with eviction; other failures fail
// the request.
bool take_built(Server& S) {
  if (S.built.empty()) return false;
  bool failed = false;
  for (const Built& b : S.built) {
    Request& r = S.reqs[b.id];
    if (b.e) {
      S.plans.insert({{b.e->N, b.e->s}, b.e});
      ++S.stats.resident_plans;
      ++S.stats.plans_built;
      S.stats.build_ms_total += b.ms;
      r.plan = b.e;
      r.build_ms = b.ms;
      S.queue.push_front(b.id);
    } else if (b.status == SFT_ENOMEM) {
      r.build_here = true;
      S.queue.push_front(b.id);
    } else {
      r.state = 3;
      r.status = b.status;
      r.t_done = Clock::now();
      ++S.stats.failed;
      failed = true;
    }
  }
  S.built.clear();
  if (failed) S.done_cv.notify_all();
  return true;
}

void CUDART_CB on_slot_done(void* p) {
  Slot* sl = static_cast<Slot*>(p);
  {
    std::lock_guard<std::mutex> g(sl->srv->mu);
    sl->t_done = Clock::now();
    sl->done = true;
  }
  sl->srv->cv.notify_all();
}

void evict(Server& S, Entry* e) {
  S.lru.erase(e->lru_it);
  auto range = S.plans.equal_range({e->N, e->s});
  for (auto it = range.first; it != range.second; ++it)
    if (it->second == e) {
      S.plans.erase(it);
      break;
    }
  free_plan(&e->P);
  delete e;
  std::lock_guard<std::mutex> g(S.mu);
  ++S.stats.plans_evicted;
  --S.stats.resident_plans;
}

// A resident idle plan for (N, s), marked busy, or nullptr.
Entry* acquire_resident(Server& S, int64_t N, int32_t s) {
  auto range = S.plans.equal_range({N, s});
  for (auto it = range.first; it != range.second; ++it) {
    Entry* e = it->second;
    if (!e->busy) {
      S.lru.erase(e->lru_it);
      e->busy = true;
      return e;
    }
  }
  return nullptr;
}

// A resident idle plan for (N, s), or a new one carved from the arena (evicting least recently
// used idle plans when it does not fit).  SFT_ENOMEM when it cannot fit beside the busy plans.
sft_status acquire(Server& S, int64_t N, int32_t s, Entry** out, bool* reused) {
  if (Entry* r = acquire_resident(S, N, s)) {
    *out = r;
    *reused = true;
    return SFT_OK;
  }
  Entry* e = new (std::nothrow) Entry();
  if (!e) return SFT_ENOMEM;
  for (;;) {
    sft_status st = build_plan(&e->P, N, s, &S.cfg.variant, 0, nullptr, 0, nullptr, 0, &S.arena);
    if (st == SFT_OK) break;
    const size_t need = e->P.want_bytes;
    free_plan(&e->P);
    e->P = Plan();
    if (st != SFT_ENOMEM || S.lru.empty()) {
      delete e;
      return st;
    }
    // evict at least one idle plan, and on until a block of this plan's size is free (builders
    // allocate concurrently, so the retry may still miss), then build again
    do {
      evict(S, S.lru.front());
    } while (!S.lru.empty() && S.arena.largest_free() < need);
  }
  e->N = N;
  e->s = s;
  e->busy = true;
  S.plans.insert({{N, s}, e});
  {
    std::lock_guard<std::mutex> g(S.mu);
    ++S.stats.resident_plans;
  }
  *out = e;
  *reused = false;
  return SFT_OK;
}

void release_plan(Server& S, Entry* e) {
  e->busy = false;
  S.lru.push_back(e);
  e->lru_it = std::prev(S.lru.end());
}

// Upload the batch's plan records, block prefixes and pointers, launch every stage, and queue the
// completion callback, all on the slot's stream.
cudaError_t launch_slot(Server& S, Slot& sl, const std::vector<Request*>& rq, int* launched) {
  const int n = (int)rq.size();
  const size_t o_prefix = align256(sizeof(DevPlan) * (size_t)n);
  const size_t o_ptrs = align256(o_prefix + sizeof(int32_t) * (size_t)kStCount * (n + 1));
  const size_t used = o_ptrs + sizeof(void*) * 4 * (size_t)n;
  if (used > sl.bytes) return cudaErrorInvalidValue;
  LaunchSet ls;
  memset(&ls, 0, sizeof(ls));
  ls.tune = S.cfg.tune;
  int32_t* pre = reinterpret_cast<int32_t*>(sl.host + o_prefix);
  void** ptr = reinterpret_cast<void**>(sl.host + o_ptrs);
  for (int i = 0; i < n; ++i) {
    const DevPlan& d = rq[i]->plan->P.d;
    memcpy(sl.host + sizeof(DevPlan) * i, &d, sizeof(DevPlan));
    ls.pmax = std::max(ls.pmax, d.pmax);
    if (d.rader) ls.rlmax = std::max(ls.rlmax, d.rLmax);
    if (d.rader) ls.rtpt = std::max(ls.rtpt, d.rTpt);
    ls.kmax = std::max(ls.kmax, d.K);
    ptr[i] = const_cast<void*>(rq[i]->f);
    ptr[n + i] = rq[i]->w;
    ptr[2 * n + i] = rq[i]->c;
    ptr[3 * n + i] = rq[i]->n;
  }
  for (int k = 0; k < kStCount; ++k) {
    int64_t acc = 0;
    for (int i = 0; i < n; ++i) {
      pre[(size_t)k * (n + 1) + i] = (int32_t)acc;
      acc += signal_blocks(rq[i]->plan->P.d, k, ls.tune);
    }
    if (acc > 0x7fffffff) return cudaErrorInvalidValue;
    pre[(size_t)k * (n + 1) + n] = (int32_t)acc;
    ls.blocks[k] = (int32_t)acc;
    ls.blk[k] = reinterpret_cast<const int32_t*>(sl.dev + o_prefix) + (size_t)k * (n + 1);
  }
  cudaError_t e = cudaMemcpyAsync(sl.dev, sl.host, used, cudaMemcpyHostToDevice, sl.st);
  if (e != cudaSuccess) return e;
  BatchView bv;
  memset(&bv, 0, sizeof(bv));
  bv.plans = reinterpret_cast<const DevPlan*>(sl.dev);
  bv.n = n;
  void** dptr = reinterpret_cast<void**>(sl.dev + o_ptrs);
  bv.f = const_cast<const void* const*>(dptr);
  bv.out_w = reinterpret_cast<int64_t* const*>(dptr + n);
  bv.out_c = reinterpret_cast<double2* const*>(dptr + 2 * n);
  bv.out_n = reinterpret_cast<int32_t* const*>(dptr + 3 * n);
  e = run_stages(rq[0]->plan->P.d, bv, ls, sl.st, nullptr, launched);
  if (e != cudaSuccess) return e;
  return cudaLaunchHostFunc(sl.st, on_slot_done, &sl);
}

// Wait on the scheduler's condition until pred() holds.  Every 20 ms without progress the busy
// slots' streams are queried (outside the lock): a stream in an error state will never run its
// completion callback, so its slot is marked dead and finished, and its requests fail.
template <typename Pred>
void wait_or_poll(Server& S, std::unique_lock<std::mutex>& lk, Pred pred) {
  while (!pred()) {
    if (S.cv.wait_for(lk, std::chrono::milliseconds(20)) != std::cv_status::timeout) continue;
    std::vector<Slot*> busy;
    for (Slot* sl : S.slots)
      if (sl->busy && !sl->done) busy.push_back(sl);
    if (busy.empty()) continue;
    lk.unlock();
    std::vector<Slot*> failed;
    for (Slot* sl : busy) {
      const cudaError_t e = cudaStreamQuery(sl->st);
      if (e != cudaSuccess && e != cudaErrorNotReady) failed.push_back(sl);
    }
    lk.lock();
    for (Slot* sl : failed) {
      sl->dead = true;
      sl->done = true;
      sl->t_done = Clock::now();
    }
  }
}

void scheduler(Server* Sp) {
  Server& S = *Sp;
  cudaSetDevice(S.device);
  std::unique_lock<std::mutex> lk(S.mu);
  for (;;) {
    take_built(S);
    if (S.abort) {
      // shutdown past its limit: fail what has not started, finish what runs, then stop
      for (std::deque<int64_t>* q : {&S.queue, &S.build_q})
        for (int64_t id : *q) {
          Request& r = S.reqs[id];
          r.state = 3;
          r.status = SFT_ETIMEOUT;
          r.t_done = Clock::now();
          ++S.stats.failed;
        }
      S.queue.clear();
      S.build_q.clear();
      S.done_cv.notify_all();
    }
    // retire finished slots
    bool retired = false;
    for (Slot* sl : S.slots) {
      if (!sl->busy || !sl->done) continue;
      for (int64_t id : sl->reqs) {
        auto it = S.reqs.find(id);
        if (it == S.reqs.end()) continue;
        it->second.t_done = sl->t_done;
        if (sl->dead) {
          it->second.state = 3;
          it->second.status = SFT_ECUDA;
          ++S.stats.failed;
        } else {
          it->second.state = 2;
          ++S.stats.completed;
        }
      }
      // plans of a failed stream may still be referenced by work the device never finished:
      // they stay out of the idle list (the server is unusable after a device fault anyway)
      if (!sl->dead)
        for (Entry* e : sl->plans) release_plan(S, e);
      sl->reqs.clear();
      sl->plans.clear();
      sl->busy = sl->done = false;
      retired = true;
    }
    if (retired) S.done_cv.notify_all();
    Slot* free_slot = nullptr;
    bool any_busy = false, any_alive = false;
    for (Slot* sl : S.slots) {
      if (sl->dead) continue;
      any_alive = true;
      if (sl->busy) any_busy = true;
      else if (!free_slot) free_slot = sl;
    }
    if (!any_alive) {
      // every stream failed: fail what is queued
      for (int64_t id : S.queue) {
        Request& r = S.reqs[id];
        r.state = 3;
        r.status = SFT_ECUDA;
        r.t_done = Clock::now();
        ++S.stats.failed;
      }
      S.queue.clear();
      S.done_cv.notify_all();
      if (S.stop && S.build_q.empty() && S.building == 0 && S.built.empty()) break;
      wait_or_poll(S, lk, [&] { return S.stop || !S.queue.empty() || !S.built.empty(); });
      continue;
    }
    const bool builds_pending = !S.build_q.empty() || S.building > 0 || !S.built.empty();
    if (S.stop && S.queue.empty() && !any_busy && !builds_pending) break;
    if (S.abort && S.queue.empty()) {
      if (!any_busy && !builds_pending) break;
      wait_or_poll(S, lk, [&] {
        if (!S.built.empty()) return true;
        for (Slot* sl : S.slots)
          if (sl->busy && sl->done) return true;
        return false;
      });
      continue;
    }
    if (!free_slot || S.queue.empty()) {
      wait_or_poll(S, lk, [&] {
        if (!S.built.empty()) return true;
        const bool pending = !S.build_q.empty() || S.building > 0;
        bool busy = false, idle = false;
        for (Slot* sl : S.slots) {
          if (sl->dead) continue;
          if (sl->busy && sl->done) return true;
          (sl->busy ? busy : idle) = true;
        }
        if (S.queue.empty()) return S.stop && !busy && !pending;
        return idle;
      });
      continue;
    }
    // take up to max_batch queued requests: first those whose plan was built for them (they need
    // no memory, and the memory their plans hold comes free only once they run), then the rest
    // in arrival order.  (Taking in arrival order alone can fill the batch with requests that
    // wait for memory held by the ready ones behind them, and nothing would ever run.)
    std::vector<int64_t> take;
    for (auto it = S.queue.begin(); it != S.queue.end() && (int)take.size() < S.cfg.max_batch;) {
      if (S.reqs[*it].plan) {
        take.push_back(*it);
        it = S.queue.erase(it);
      } else {
        ++it;
      }
    }
    while (!S.queue.empty() && (int)take.size() < S.cfg.max_batch) {
      take.push_back(S.queue.front());
      S.queue.pop_front();
    }
    std::vector<Request*> rq;
    for (int64_t id : take) rq.push_back(&S.reqs[id]);   // records stay put until released
    // arena memory that will come free: plans of running batches, of requests whose plan was
    // built for them and waits to run, and of builds in flight
    bool held = any_busy || S.building > 0 || !S.build_q.empty() || !S.built.empty();
    for (Request* r : rq) held = held || r->plan != nullptr;
    for (int64_t id : S.queue) held = held || S.reqs[id].plan != nullptr;
    // Claim the slot before its work exists: its completion callback may fire before this thread
    // takes the lock again, and must find the slot busy with `done` clear so the completion is
    // not overwritten.
    free_slot->busy = true;
    free_slot->done = false;
    free_slot->reqs.clear();
    free_slot->plans.clear();
    lk.unlock();

    std::vector<int64_t> admitted, deferred, to_build;
    std::vector<Request*> arq;
    std::vector<std::pair<int64_t, sft_status>> failed;
    std::vector<int32_t> was_reused;
    int64_t built = 0, reused_n = 0;
    double built_ms = 0.0;
    for (size_t i = 0; i < take.size(); ++i) {
      if (rq[i]->plan) {                       // a builder made its plan: it joins this batch
        was_reused.push_back(0);
        admitted.push_back(take[i]);
        arq.push_back(rq[i]);
        continue;
      }
      if (!deferred.empty()) {                 // keep arrival order behind a waiting request
        deferred.push_back(take[i]);
        continue;
      }
      if (S.cfg.build_threads > 0 && !rq[i]->build_here) {
        if (Entry* e = acquire_resident(S, rq[i]->N, rq[i]->s)) {
          rq[i]->plan = e;
          ++reused_n;
          was_reused.push_back(1);
          admitted.push_back(take[i]);
          arq.push_back(rq[i]);
        } else {
          to_build.push_back(take[i]);         // built beside the scheduler; later batches
        }
        continue;
      }
      Entry* e = nullptr;
      bool reused = false;
      const auto tb = Clock::now();
      const sft_status st = acquire(S, rq[i]->N, rq[i]->s, &e, &reused);
      if (st == SFT_OK) {
        rq[i]->plan = e;                       // read only by this thread until retired
        if (!reused) {
          rq[i]->build_ms = ms_between(tb, Clock::now());
          built_ms += rq[i]->build_ms;
        }
        (reused ? reused_n : built) += 1;
        was_reused.push_back(reused ? 1 : 0);
        admitted.push_back(take[i]);
        arq.push_back(rq[i]);
      } else if (st == SFT_ENOMEM && (held || !admitted.empty())) {
        deferred.push_back(take[i]);           // memory frees up when running work finishes
      } else {
        failed.push_back({take[i], st});
      }
    }
    // keep room for the builders: idle plans, least recently used first, go until a quarter of
    // the budget is free in one block (a stream of new lengths otherwise fills the arena with
    // plans that are not used again, and every build would fall back to the scheduler)
    if (!to_build.empty())
      while (!S.lru.empty() && S.arena.largest_free() < S.cfg.mem_budget / 4) evict(S, S.lru.front());
    int launched = 0;
    cudaError_t ce = cudaSuccess;
    if (!arq.empty()) ce = launch_slot(S, *free_slot, arq, &launched);

    lk.lock();
    for (auto it = deferred.rbegin(); it != deferred.rend(); ++it) S.queue.push_front(*it);
    if (!to_build.empty()) {
      for (int64_t id : to_build) S.build_q.push_back(id);
      S.build_cv.notify_all();
    }
    S.stats.build_ms_total += built_ms;
    for (auto& f : failed) {
      Request& r = S.reqs[f.first];
      r.state = 3;
      r.status = f.second;
      r.t_done = Clock::now();
      ++S.stats.failed;
    }
    S.stats.plans_built += built;
    S.stats.plans_reused += reused_n;
    if (!arq.empty()) {
      const auto now = Clock::now();
      for (size_t i = 0; i < arq.size(); ++i) {
        arq[i]->batch_size = (int32_t)arq.size();
        arq[i]->reused = was_reused[i];
      }
      if (ce == cudaSuccess) {
        // busy since the claim; `done` may already be set by the completion callback
        free_slot->reqs = admitted;
        for (Request* r : arq) {
          r->state = 1;
          r->t_launch = now;
          free_slot->plans.push_back(r->plan);
        }
        ++S.stats.batches;
        S.stats.kernel_launches += launched;
        S.stats.max_batch_seen = std::max(S.stats.max_batch_seen, (int32_t)arq.size());
      } else {
        cudaGetLastError();
        free_slot->busy = free_slot->done = false;
        for (Request* r : arq) {
          r->state = 3;
          r->status = SFT_ECUDA;
          r->t_done = now;
          release_plan(S, r->plan);
          ++S.stats.failed;
        }
      }
    } else {
      free_slot->busy = free_slot->done = false;      // nothing was launched: release the claim
    }
    if (!failed.empty() || ce != cudaSuccess) S.done_cv.notify_all();
    if (arq.empty() && !deferred.empty()) {
      // nothing could start: wait for running work or a build to finish (either frees memory
      // or brings a plan)
      wait_or_poll(S, lk, [&] {
        if (!S.built.empty()) return true;
        bool busy = false;
        for (Slot* sl : S.slots) {
          if (sl->busy && sl->done) return true;
          busy = busy || sl->busy;
        }
        return !busy && S.building == 0 && S.build_q.empty();
      });
    }
  }
  S.exited = true;
  S.exit_cv.notify_all();
}

void destroy_server(Server* S) {
  for (Slot* sl : S->slots) {
    if (sl->st) cudaStreamDestroy(sl->st);
    if (sl->dev) cudaFree(sl->dev);
    if (sl->host) cudaFreeHost(sl->host);
    delete sl;
  }
  S->slots.clear();
  for (auto& kv : S->plans) {
    free_plan(&kv.second->P);
    delete kv.second;
  }
  S->plans.clear();
  S->lru.clear();
}

}  // namespace
}  // namespace sft

struct sft_server_s {
  sft::Server S;
};

extern "C" {

void sft_server_config_init(sft_server_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->mem_budget = (size_t)8 << 30;
  cfg->max_batch = 64;
  cfg->max_inflight = 2;
  cfg->build_threads = 2;
  sft_variant_init(&cfg->variant);
  cfg->tune = sft::default_tuning();
}

sft_status sft_server_create(sft_server_t* out, const sft_server_config* cfg) {
  return sft::guarded("sft_server_create", [&]() -> sft_status {
    using namespace sft;
    if (!out || !cfg) { set_error("sft_server_create: NULL argument"); return SFT_EINVAL; }
    *out = nullptr;
    if (cfg->mem_budget < ((size_t)1 << 20) || cfg->max_batch < 1 || cfg->max_batch > kMaxServerBatch ||
        cfg->max_inflight < 1 || cfg->max_inflight > kMaxInflight || cfg->build_threads < 0 ||
        cfg->build_threads > kMaxBuilders) {
      set_error("sft_server_create: need mem_budget >= 1 MiB, 1 <= max_batch <= 256, "
                "1 <= max_inflight <= 8, 0 <= build_threads <= 16");
      return SFT_EINVAL;
    }
    sft_tuning tune = cfg->tune.resample_threads == 0 ? default_tuning() : cfg->tune;
    std::string why;
    if (!tuning_valid(tune, &why)) { set_error("sft_server_create: " + why); return SFT_EINVAL; }
    sft_server_s* h = new (std::nothrow) sft_server_s();
    if (!h) { set_error("host allocation failed"); return SFT_ENOMEM; }
    Server& S = h->S;
    S.cfg = *cfg;
    S.cfg.tune = tune;
    memset(&S.stats, 0, sizeof(S.stats));
    cudaGetDevice(&S.device);
    cudaError_t e = S.arena.init(cfg->mem_budget);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete h;
      set_error(std::string("sft_server_create: arena allocation failed: ") + cudaGetErrorString(e));
      return SFT_ENOMEM;
    }
    const int nb = cfg->max_batch;
    const size_t slot_bytes = align256(align256(sizeof(DevPlan) * (size_t)nb) +
                                       sizeof(int32_t) * (size_t)kStCount * (nb + 1)) +
                              sizeof(void*) * 4 * (size_t)nb;
    for (int i = 0; i < cfg->max_inflight && e == cudaSuccess; ++i) {
      Slot* sl = new (std::nothrow) Slot();
      if (!sl) { e = cudaErrorMemoryAllocation; break; }
      sl->srv = &S;
      sl->bytes = slot_bytes;
      S.slots.push_back(sl);
      e = cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = dev_malloc((void**)&sl->dev, slot_bytes);
      if (e == cudaSuccess) e = host_alloc((void**)&sl->host, slot_bytes);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      destroy_server(&S);
      delete h;
      set_error(std::string("sft_server_create: set-up failed: ") + cudaGetErrorString(e));
      return SFT_ENOMEM;
    }
    S.th = std::thread(scheduler, &S);
    for (int i = 0; i < cfg->build_threads; ++i) S.builders.emplace_back(builder, &S);
    *out = h;
    return SFT_OK;
  });
}

sft_status sft_server_submit(sft_server_t server, int64_t N, int32_t s, const void* f_dev,
                             int64_t* out_freqs_dev, void* out_coefs_dev, int32_t* out_count_dev,
                             sft_request_t* id) {
  return sft::guarded("sft_server_submit", [&]() -> sft_status {
    using namespace sft;
    if (!server || !f_dev || !out_freqs_dev || !out_coefs_dev || !out_count_dev || !id) {
      set_error("sft_server_submit: NULL argument");
      return SFT_EINVAL;
    }
    Server& S = server->S;
    const size_t align = S.cfg.variant.input == SFT_IN_C64 ? 8 : 16;
    if ((uintptr_t)f_dev % align) { set_error("sft_server_submit: f is misaligned"); return SFT_EINVAL; }
    {
      std::lock_guard<std::mutex> g(S.mu);
      if (S.stop) { set_error("sft_server_submit: the server is stopping"); return SFT_EINVAL; }
      const int64_t rid = S.next_id++;
      Request& r = S.reqs[rid];
      r.N = N;
      r.s = s;
      r.f = f_dev;
      r.w = out_freqs_dev;
      r.c = out_coefs_dev;
      r.n = out_count_dev;
      r.t_submit = Clock::now();
      S.queue.push_back(rid);
      ++S.stats.submitted;
      *id = rid;
    }
    S.cv.notify_all();
    return SFT_OK;
  });
}

sft_status sft_server_query(sft_server_t server, sft_request_t id, sft_request_info* info) {
  using namespace sft;
  if (!server || !info) { set_error("sft_server_query: NULL argument"); return SFT_EINVAL; }
  Server& S = server->S;
  std::lock_guard<std::mutex> g(S.mu);
  auto it = S.reqs.find(id);
  if (it == S.reqs.end()) { set_error("sft_server_query: unknown request"); return SFT_EINVAL; }
  const Request& r = it->second;
  memset(info, 0, sizeof(*info));
  info->state = r.state;
  info->status = r.status;
  info->batch_size = r.batch_size;
  info->plan_reused = r.reused;
  if (r.state >= 1 && r.state != 3) info->queued_ms = ms_between(r.t_submit, r.t_launch);
  if (r.state >= 2) info->latency_ms = ms_between(r.t_submit, r.t_done);
  info->build_ms = r.build_ms;
  return SFT_OK;
}

sft_status sft_server_poll(sft_server_t server, sft_request_t id, int32_t* done) {
  if (!done) { sft::set_error("sft_server_poll: NULL argument"); return SFT_EINVAL; }
  *done = 0;
  sft_request_info info;
  const sft_status s = sft_server_query(server, id, &info);
  if (s != SFT_OK) return s;
  *done = info.state >= 2 ? 1 : 0;
  return info.state == 3 ? (sft_status)info.status : SFT_OK;
}

sft_status sft_server_wait(sft_server_t server, sft_request_t id, int32_t timeout_ms) {
  using namespace sft;
  if (!server) { set_error("sft_server_wait: NULL server"); return SFT_EINVAL; }
  Server& S = server->S;
  std::unique_lock<std::mutex> lk(S.mu);
  auto it = S.reqs.find(id);
  if (it == S.reqs.end()) { set_error("sft_server_wait: unknown request"); return SFT_EINVAL; }
  auto finished = [&] {
    auto jt = S.reqs.find(id);
    return jt == S.reqs.end() || jt->second.state >= 2;
  };
  if (timeout_ms < 0) {
    S.done_cv.wait(lk, finished);
  } else if (!S.done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished)) {
    set_error("sft_server_wait: timed out");
    return SFT_ETIMEOUT;
  }
  return SFT_OK;
}

sft_status sft_server_release(sft_server_t server, sft_request_t id) {
  using namespace sft;
  if (!server) { set_error("sft_server_release: NULL server"); return SFT_EINVAL; }
  Server& S = server->S;
  std::lock_guard<std::mutex> g(S.mu);
  auto it = S.reqs.find(id);
  if (it == S.reqs.end()) { set_error("sft_server_release: unknown request"); return SFT_EINVAL; }
  if (it->second.state < 2) { set_error("sft_server_release: request not finished"); return SFT_EBUSY; }
  S.reqs.erase(it);
  return SFT_OK;
}

sft_status sft_server_stats_read(sft_server_t server, sft_server_stats* out) {
  using namespace sft;
  if (!server || !out) { set_error("sft_server_stats_read: NULL argument"); return SFT_EINVAL; }
  Server& S = server->S;
  {
    std::lock_guard<std::mutex> g(S.mu);
    *out = S.stats;
  }
  S.arena.usage(&out->arena_bytes, &out->arena_used, &out->arena_peak);
  return SFT_OK;
}

sft_status sft_server_destroy(sft_server_t server) {
  using namespace sft;
  if (!server) return SFT_OK;
  Server& S = server->S;
  {
    std::lock_guard<std::mutex> g(S.mu);
    S.stop = true;
  }
  S.cv.notify_all();
  {
    // queued and running requests finish; past a minute without the scheduler exiting, what has
    // not started fails (SFT_ETIMEOUT) and the scheduler stops after the running work
    std::unique_lock<std::mutex> lk(S.mu);
    if (!S.exit_cv.wait_for(lk, std::chrono::seconds(60), [&] { return S.exited; })) {
      S.abort = true;
      S.cv.notify_all();
    }
  }
  if (S.th.joinable()) S.th.join();
  {
    std::lock_guard<std::mutex> g(S.mu);
    S.stop_builders = true;
  }
  S.build_cv.notify_all();
  for (std::thread& t : S.builders)
    if (t.joinable()) t.join();
  // plans a builder finished after an aborted scheduler stopped were never made resident
  for (Built& b : S.built)
    if (b.e) {
      free_plan(&b.e->P);
      delete b.e;
    }
  S.built.clear();
  destroy_server(&S);
  delete server;
  return SFT_OK;
}

}  // extern "C"
