// Host check of the serving scheduler (serve_sched.h) with a fake executor:
// builds and solves sleep for the times a scenario gives and report the
// bytes it gives, while the executor records, independently of the
// scheduler's own counters, how many requests run at once, the device bytes
// held at any moment (live factorisations + running requests' work) and the
// order in which requests start.  Usage: serve_check <scenario>; prints
// "name value" lines.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "serve_sched.h"

using namespace hf::serve;

struct FakeReq {
  int tag;
  double build_ms, solve_ms;
  size_t fac_bytes, work_bytes;
  int solve_status = 0;
};

struct FakeExec : Executor {
  std::mutex mu;
  int running = 0, peak_running = 0;
  size_t live_fac = 0, run_work = 0, peak_held = 0;
  std::vector<int> start_order;
  std::map<int, int> handles;   // live handles (id -> tag)
  int next_handle = 1;
  int builds = 0, solves = 0;
  bool concurrent_same_key = false;
  std::map<uint64_t, int> key_running;

  void enter(Request& r, size_t work) {
    std::lock_guard<std::mutex> lk(mu);
    ++running;
    if (running > peak_running) peak_running = running;
    run_work += work;
    if (live_fac + run_work > peak_held) peak_held = live_fac + run_work;
    if (key_running[r.key]++ > 0) concurrent_same_key = true;
  }
  void leave(Request& r, size_t work) {
    std::lock_guard<std::mutex> lk(mu);
    --running;
    run_work -= work;
    --key_running[r.key];
  }
  static void sleep_ms(double ms) {
    std::this_thread::sleep_for(std::chrono::microseconds((long long)(ms * 1000)));
  }
  int build(int, Request& r, void** handle, size_t* bytes) override {
    auto* q = static_cast<FakeReq*>(r.payload);
    {
      std::lock_guard<std::mutex> lk(mu);
      start_order.push_back(q->tag);
      ++builds;
    }
    enter(r, q->work_bytes);
    sleep_ms(q->build_ms);
    {
      std::lock_guard<std::mutex> lk(mu);
      live_fac += q->fac_bytes;
      if (live_fac + run_work > peak_held) peak_held = live_fac + run_work;
      int id = next_handle++;
      handles[id] = q->tag;
      *handle = reinterpret_cast<void*>((intptr_t)id);
    }
    *bytes = q->fac_bytes;
    return 0;
  }
  int solve(int, Request& r, void* handle, size_t* bytes) override {
    auto* q = static_cast<FakeReq*>(r.payload);
    if (r.reused) {
      std::lock_guard<std::mutex> lk(mu);
      start_order.push_back(q->tag);
    }
    if (r.reused) enter(r, q->work_bytes);
    sleep_ms(q->solve_ms);
    leave(r, q->work_bytes);
    {
      std::lock_guard<std::mutex> lk(mu);
      ++solves;
    }
    (void)handle;
    *bytes = q->fac_bytes;
    return q->solve_status;
  }
  bool reusable_after(int status) override { return status == 0; }
  void release(void* handle) override {
    std::lock_guard<std::mutex> lk(mu);
    int id = (int)reinterpret_cast<intptr_t>(handle);
    (void)id;
    handles.erase(id);
    // every fake factorisation of a scenario has the same size
    live_fac -= fac_size;
  }
  void release_payload(Request& r) override {
    delete static_cast<FakeReq*>(r.payload);
    r.payload = nullptr;
  }
  size_t fac_size = 0;
};

static std::unique_ptr<Request> req(int tag, uint64_t key, double build_ms, double solve_ms,
                                    size_t fac, size_t work) {
  auto r = std::make_unique<Request>();
  r->key = key;
  r->sig = {(double)key};
  r->est_build = fac;
  r->est_work = work;
  r->payload = new FakeReq{tag, build_ms, solve_ms, fac, work};
  return r;
}

static void report(const char* name, Scheduler& s, FakeExec& ex, const std::vector<Done>& done) {
  auto c = s.counters();
  std::printf("scenario %s\n", name);
  std::printf("budget %zu\n", c.budget);
  std::printf("sched_peak_bytes %zu\n", c.peak_bytes);
  std::printf("exec_peak_held %zu\n", ex.peak_held);
  std::printf("sched_peak_running %d\n", c.peak_running);
  std::printf("exec_peak_running %d\n", ex.peak_running);
  std::printf("builds %lld\n", (long long)c.builds);
  std::printf("reuses %lld\n", (long long)c.reuses);
  std::printf("evictions %lld\n", (long long)c.evictions);
  std::printf("rejected %lld\n", (long long)c.rejected);
  std::printf("concurrent_same_key %d\n", ex.concurrent_same_key ? 1 : 0);
  std::printf("live_handles_after_shutdown %zu\n", ex.handles.size());
  std::printf("start_order");
  for (int t : ex.start_order) std::printf(" %d", t);
  std::printf("\n");
  int ok = 0, oom = 0;
  for (auto& d : done) (d.status == 0 ? ok : oom) += 1;
  std::printf("done_ok %d\ndone_oom %d\n", ok, oom);
}

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  std::string sc = argv[1];
  FakeExec ex;
  std::vector<Done> done;
  auto run = [&](Scheduler& s) {
    s.drain();
    done = s.poll(0);
  };
  if (sc == "overlap") {
    // 8 slots, 16 independent requests, ample memory: 8 run at once
    ex.fac_size = 10;
    Scheduler s(&ex, 8, 1000000, 0, 2);
    for (int i = 0; i < 16; ++i) s.submit(req(i, 100 + i, 5, 40, 10, 5));
    run(s);
    s.shutdown();
    report("overlap", s, ex, done);
  } else if (sc == "backpressure") {
    // 4 slots but the budget holds one request at a time
    ex.fac_size = 40;
    Scheduler s(&ex, 4, 70, 0, 2);
    for (int i = 0; i < 6; ++i) s.submit(req(i, 200 + i, 5, 10, 40, 20));
    run(s);
    s.shutdown();
    report("backpressure", s, ex, done);
  } else if (sc == "oom") {
    // a request larger than the whole budget is rejected; the others run
    ex.fac_size = 40;
    Scheduler s(&ex, 2, 100, 0, 2);
    s.submit(req(0, 300, 5, 5, 40, 10));
    s.submit(req(1, 301, 5, 5, 90, 30));
    s.submit(req(2, 302, 5, 5, 40, 10));
    run(s);
    s.shutdown();
    report("oom", s, ex, done);
  } else if (sc == "reuse") {
    // five requests on one operator: built once, reused, never concurrent
    ex.fac_size = 30;
    Scheduler s(&ex, 4, 1000, 8, 2);
    for (int i = 0; i < 5; ++i) s.submit(req(i, 400, 20, 10, 30, 5));
    run(s);
    s.shutdown();
    report("reuse", s, ex, done);
  } else if (sc == "evict") {
    // idle factorisations are evicted (least recently used first) only when
    // a new request needs their memory; A, B, C in turn, then A again
    ex.fac_size = 40;
    Scheduler s(&ex, 1, 100, 8, 2);
    s.submit(req(0, 501, 2, 2, 40, 10));   // A
    s.submit(req(1, 502, 2, 2, 40, 10));   // B: fits beside A
    s.submit(req(2, 503, 2, 2, 40, 10));   // C: evicts A
    s.submit(req(3, 502, 2, 2, 40, 10));   // B again: reused
    s.submit(req(4, 501, 2, 2, 40, 10));   // A again: rebuilt, evicts C
    run(s);
    s.shutdown();
    report("evict", s, ex, done);
  } else if (sc == "fifo") {
    // a request waiting for memory is not overtaken by a later small one
    ex.fac_size = 0;
    Scheduler s(&ex, 4, 100, 0, 2);
    s.submit(req(0, 601, 1, 60, 0, 70));   // holds 70 for 60 ms
    std::this_thread::sleep_for(std::chrono::milliseconds(10));
    s.submit(req(1, 602, 1, 5, 0, 60));    // must wait for 0
    s.submit(req(2, 603, 1, 5, 0, 10));    // would fit now, must not overtake 1
    run(s);
    s.shutdown();
    report("fifo", s, ex, done);
  } else if (sc == "drop") {
    // a factorisation whose solve failed is not kept: the next request of the
    // same operator builds a new one
    ex.fac_size = 20;
    Scheduler s(&ex, 1, 1000, 8, 2);
    auto a = req(0, 700, 2, 2, 20, 5);
    static_cast<FakeReq*>(a->payload)->solve_status = 6;
    s.submit(std::move(a));
    s.submit(req(1, 700, 2, 2, 20, 5));
    s.submit(req(2, 700, 2, 2, 20, 5));
    run(s);
    s.shutdown();
    report("drop", s, ex, done);
  } else {
    return 2;
  }
  return 0;
}
