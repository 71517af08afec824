// Request scheduler of the serving loop: admission of solve requests into a
// fixed number of slots under a device-memory budget, with a cache of
// resident factorisations reused by later requests of the same problem.
//
// This header holds no CUDA code: the work itself is done by an Executor
// (the CUDA one lives in serve.cpp; the host tests drive a fake one), so the
// admission, back-pressure and reuse rules can be checked without a GPU.
//
// Rules.
//  * Slots: `slots` worker threads; each takes one request at a time.  An
//    idle worker scans the queue in arrival order and takes the first
//    request it may admit; requests that arrive while others run are
//    admitted as soon as a slot and memory are free.
//  * Memory: resident factorisations + admitted requests' estimates never
//    exceed the budget.  To admit a request, unused cached factorisations
//    are evicted (least recently used first), but only when that makes the
//    request fit.  A request that does not fit stops the scan (later ones
//    may not overtake it), except when nothing is running or resident-in-
//    use at all: then it can never fit and completes with HFSEM_ERR_OOM.
//  * Reuse: requests carry a key (a hash of everything the factorisation
//    depends on, with the full signature compared on a hash match).  A
//    request whose factorisation is resident and idle takes it (exclusive
//    use while it runs); one whose factorisation is in use, or being built
//    by an admitted request, waits and is skipped by the scan.
//  * Cache: after a request, its factorisation stays resident (idle) while
//    at most `cache_entries` idle ones are kept; beyond that the least
//    recently used idle one is released.
#pragma once

#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace hf {
namespace serve {

struct Entry {                  // a resident factorisation
  uint64_t key = 0;
  std::vector<double> sig;      // full signature (compared on a key match)
  void* handle = nullptr;       // executor-owned
  size_t bytes = 0;             // device bytes it holds
  bool in_use = false;
  std::list<Entry*>::iterator lru_it;
  bool in_lru = false;
};

struct Request {
  int64_t id = 0;
  uint64_t key = 0;
  std::vector<double> sig;
  size_t est_build = 0;         // estimated bytes of a new factorisation
  size_t est_work = 0;          // estimated bytes of the solve's work space
  void* payload = nullptr;      // executor-owned request data
  double t_submit = 0, t_start = 0, t_done = 0;
  int status = 0;
  int reused = 0;
  std::string msg;
};

struct Done {
  int64_t id;
  int status;
  int reused;
  double t_submit, t_start, t_done;
  std::string msg;
};

// The work: build a factorisation for a request, solve a request with one,
// release one.  Called from worker threads, outside the scheduler's lock.
struct Executor {
  virtual ~Executor() {}
  virtual void thread_init(int slot) { (void)slot; }
  virtual void thread_exit(int slot) { (void)slot; }
  // build: the executor's handle and its device bytes; status != 0 on
  // failure (then no handle).  solve: the handle's device bytes afterwards
  // (its work space grows with the right-hand sides it has served)
  virtual int build(int slot, Request& r, void** handle, size_t* bytes) = 0;
  virtual int solve(int slot, Request& r, void* handle, size_t* bytes) = 0;
  virtual void release(void* handle) = 0;
  virtual void release_payload(Request& r) = 0;
  // whether a factorisation may serve later requests after a solve that
  // returned `status` (a device failure leaves it untrusted)
  virtual bool reusable_after(int status) { (void)status; return true; }
};

class Scheduler {
 public:
  Scheduler(Executor* ex, int slots, size_t budget, int cache_entries, int oom_status)
      : ex_(ex), slots_(slots), budget_(budget), cache_cap_(cache_entries), oom_(oom_status),
        t0_(std::chrono::steady_clock::now()) {
    for (int s = 0; s < slots_; ++s) workers_.emplace_back([this, s] { work(s); });
  }

  ~Scheduler() { shutdown(); }

  void shutdown() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      if (stopped_) return;
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : workers_) t.join();
    std::lock_guard<std::mutex> lk(mu_);
    for (auto& r : queue_) {
      ex_->release_payload(*r);
    }
    queue_.clear();
    for (auto* e : released_)
      if (e) {
        ex_->release(e->handle);
        delete e;
      }
    released_.clear();
    for (void* h : drop_handles_) ex_->release(h);
    drop_handles_.clear();
    for (auto& kv : cache_) {
      ex_->release(kv.second->handle);
      delete kv.second;
    }
    cache_.clear();
    lru_.clear();
    stopped_ = true;
  }

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0_).count();
  }

  int64_t submit(std::unique_ptr<Request> r) {
    std::lock_guard<std::mutex> lk(mu_);
    r->id = next_id_++;
    r->t_submit = now();
    int64_t id = r->id;
    queue_.push_back(std::move(r));
    ++outstanding_;
    cv_.notify_all();
    return id;
  }

  // completed requests since the last call, at most max (all if max <= 0)
  std::vector<Done> poll(int max) {
    std::lock_guard<std::mutex> lk(mu_);
    std::vector<Done> out;
    while (!done_.empty() && (max <= 0 || (int)out.size() < max)) {
      out.push_back(std::move(done_.front()));
      done_.pop_front();
    }
    return out;
  }

  // block until every submitted request has completed
  void drain() {
    std::unique_lock<std::mutex> lk(mu_);
    cv_done_.wait(lk, [this] { return outstanding_ == 0; });
  }

  struct Counters {
    size_t resident = 0, inflight = 0, budget = 0, peak_bytes = 0;
    int running = 0, peak_running = 0, cached = 0, queued = 0;
    int64_t builds = 0, reuses = 0, evictions = 0, rejected = 0;
  };
  Counters counters() {
    std::lock_guard<std::mutex> lk(mu_);
    Counters c;
    c.resident = resident_;
    c.inflight = inflight_;
    c.budget = budget_;
    c.peak_bytes = peak_bytes_;
    c.running = running_;
    c.peak_running = peak_running_;
    c.cached = (int)cache_.size();
    c.queued = (int)queue_.size();
    c.builds = builds_;
    c.reuses = reuses_;
    c.evictions = evictions_;
    c.rejected = rejected_;
    return c;
  }

 private:
  Entry* find(const Request& r) {
    auto range = cache_.equal_range(r.key);
    for (auto it = range.first; it != range.second; ++it)
      if (it->second->sig == r.sig) return it->second;
    return nullptr;
  }
  bool building(const Request& r) const {
    for (auto& b : building_)
      if (b.first == r.key && *b.second == r.sig) return true;
    return false;
  }
  size_t idle_bytes(const Entry* keep) const {
    size_t b = 0;
    for (auto* e : lru_)
      if (e != keep) b += e->bytes;
    return b;
  }
  void drop(Entry* e) {   // an idle entry leaves the cache (lock held)
    if (e->in_lru) lru_.erase(e->lru_it);
    auto range = cache_.equal_range(e->key);
    for (auto it = range.first; it != range.second; ++it)
      if (it->second == e) {
        cache_.erase(it);
        break;
      }
    resident_ -= e->bytes;
    released_.push_back(e);
  }
  void note_peak() {
    if (resident_ + inflight_ > peak_bytes_) peak_bytes_ = resident_ + inflight_;
    if (running_ > peak_running_) peak_running_ = running_;
  }
  void finish(std::unique_ptr<Request> r) {   // lock held
    Done d{r->id, r->status, r->reused, r->t_submit, r->t_start, r->t_done, r->msg};
    ex_->release_payload(*r);
    done_.push_back(std::move(d));
    --outstanding_;
    cv_done_.notify_all();
  }

  // Pick the next request this worker may run (lock held).  Returns it with
  // its cache entry (nullptr: build a new one).
  std::unique_ptr<Request> pick(Entry** hit) {
    for (auto it = queue_.begin(); it != queue_.end();) {
      Request& r = **it;
      Entry* e = find(r);
      if ((e && e->in_use) || (!e && building(r))) {
        ++it;                  // its factorisation is busy: let it wait
        continue;
      }
      size_t need = r.est_work + (e ? 0 : r.est_build);
      size_t free_now = budget_ > resident_ + inflight_ ? budget_ - resident_ - inflight_ : 0;
      if (need > free_now && need <= free_now + idle_bytes(e)) {
        // evict idle factorisations, least recently used first
        for (auto l = lru_.begin(); l != lru_.end() && need > free_now;) {
          Entry* v = *l;
          ++l;
          if (v == e) continue;
          drop(v);
          ++evictions_;
          free_now = budget_ > resident_ + inflight_ ? budget_ - resident_ - inflight_ : 0;
        }
      }
      if (need <= free_now) {
        std::unique_ptr<Request> out = std::move(*it);
        queue_.erase(it);
        *hit = e;
        if (e) {
          e->in_use = true;
          if (e->in_lru) {
            lru_.erase(e->lru_it);
            e->in_lru = false;
          }
        }
        inflight_ += need;
        return out;
      }
      bool anything_held = running_ > 0;
      for (auto& kv : cache_) anything_held = anything_held || kv.second->in_use;
      if (!anything_held) {
        // nothing else holds memory and evicting every idle factorisation
        // is not enough: it can never fit
        std::unique_ptr<Request> out = std::move(*it);
        it = queue_.erase(it);
        out->status = oom_;
        out->msg = "request needs more device memory than the server's budget";
        out->t_start = out->t_done = now();
        ++rejected_;
        finish(std::move(out));
        continue;
      }
      break;                   // memory-blocked: later requests may not overtake it
    }
    return nullptr;
  }

  void flush_released() {      // release dropped entries outside the lock
    std::vector<Entry*> rel;
    std::vector<void*> hs;
    {
      std::lock_guard<std::mutex> lk(mu_);
      rel.swap(released_);
      hs.swap(drop_handles_);
    }
    for (auto* e : rel) {
      if (!e) continue;
      ex_->release(e->handle);
      delete e;
    }
    for (void* h : hs) ex_->release(h);
  }

  void work(int slot) {
    ex_->thread_init(slot);
    for (;;) {
      std::unique_ptr<Request> r;
      Entry* e = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] {
          if (stop_) return true;
          r = pick(&e);
          return r != nullptr;
        });
        if (!r) break;
        ++running_;
        if (!e) building_.emplace_back(r->key, &r->sig);
        note_peak();
        r->t_start = now();
      }
      flush_released();
      const size_t charged = r->est_work + (e ? 0 : r->est_build);
      size_t fac_bytes = e ? e->bytes : 0, work_bytes = 0;
      void* handle = e ? e->handle : nullptr;
      int st = 0;
      if (!e) {
        st = ex_->build(slot, *r, &handle, &fac_bytes);
        r->reused = 0;
      } else {
        r->reused = 1;
      }
      if (st == 0) st = ex_->solve(slot, *r, handle, &work_bytes);
      if (handle && work_bytes < fac_bytes) work_bytes = fac_bytes;
      r->status = st;
      r->t_done = now();
      {
        std::lock_guard<std::mutex> lk(mu_);
        inflight_ -= charged;
        --running_;
        if (!e) {
          for (auto b = building_.begin(); b != building_.end(); ++b)
            if (b->second == &r->sig) {
              building_.erase(b);
              break;
            }
          if (handle && !ex_->reusable_after(st)) {
            drop_handles_.push_back(handle);
            handle = nullptr;
          }
          if (handle) {
            ++builds_;
            e = new Entry;
            e->key = r->key;
            e->sig = r->sig;
            e->handle = handle;
            e->bytes = work_bytes;
            cache_.emplace(e->key, e);
            resident_ += e->bytes;
          }
        } else {
          ++reuses_;
          resident_ += work_bytes - e->bytes;
          e->bytes = work_bytes;
          if (!ex_->reusable_after(st)) {
            e->in_use = false;
            drop(e);            // leaves the cache; released below
            e = nullptr;
          }
        }
        if (e) {
          e->in_use = false;
          lru_.push_back(e);
          e->lru_it = std::prev(lru_.end());
          e->in_lru = true;
          while ((int)lru_.size() > cache_cap_) drop(lru_.front());
        }
        note_peak();
        finish(std::move(r));
      }
      flush_released();
      cv_.notify_all();
    }
    ex_->thread_exit(slot);
  }

  Executor* ex_;
  int slots_;
  size_t budget_;
  int cache_cap_;
  int oom_;
  std::chrono::steady_clock::time_point t0_;
  std::mutex mu_;
  std::condition_variable cv_, cv_done_;
  std::deque<std::unique_ptr<Request>> queue_;
  std::multimap<uint64_t, Entry*> cache_;
  std::list<Entry*> lru_;                 // idle entries, least recent first
  std::vector<std::pair<uint64_t, const std::vector<double>*>> building_;
  std::vector<Entry*> released_;
  std::vector<void*> drop_handles_;     // built, never cached (failed solve)
  std::deque<Done> done_;
  std::vector<std::thread> workers_;
  size_t resident_ = 0, inflight_ = 0, peak_bytes_ = 0;
  int running_ = 0, peak_running_ = 0;
  int64_t next_id_ = 1, outstanding_ = 0;
  int64_t builds_ = 0, reuses_ = 0, evictions_ = 0, rejected_ = 0;
  bool stop_ = false, stopped_ = false;
};

}  // namespace serve
}  // namespace hf
