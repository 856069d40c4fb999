// Host-side scheduler of the serving loop (pure C++; no CUDA here, so its admission,
// batching, queueing, timeout and cancellation logic can be exercised without a GPU).
//
// Continuous batching in two phases.  Each lane (on the GPU: a CUDA stream with its own
// request workspaces) is a worker that takes a batch of the oldest pending requests (up to
// one per workspace) and runs phase A, the work that fixes a request's true memory need
// (on the GPU: its projection, which counts its tile instances).  Admission then grants
// each request a range of a fixed arena (the instance buffers, sized once from the budget)
// in arrival order; a request that does not fit goes back to the head of the queue, and
// once it has waited longer than the aging limit nothing behind it is admitted before it,
// so a large request is never overtaken forever.  Phase B launches the admitted requests
// together (on the GPU: one persistent raster launch for all of them); the worker waits for
// them, publishes their results, frees their arena ranges and takes the next batch.  Lanes
// run independently, so several batches are on the device at once, and requests that
// arrive meanwhile join the next batch of the first lane that frees up.
#pragma once

#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <functional>
#include <iterator>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

namespace gs_serve {

// First-fit allocator of ranges [offset, offset + n) of an arena of `capacity` units.
class Arena {
 public:
  explicit Arena(int64_t capacity = 0) { reset(capacity); }
  void reset(int64_t capacity) {
    cap_ = capacity > 0 ? capacity : 0;
    used_ = 0;
    free_.clear();
    if (cap_ > 0) free_[0] = cap_;
  }
  int64_t capacity() const { return cap_; }
  int64_t used() const { return used_; }
  // Offset of a free range of n units (0 for n <= 0, which takes nothing), or -1.
  int64_t alloc(int64_t n) {
    if (n <= 0) return 0;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const int64_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > n) free_[off + n] = len - n;
      used_ += n;
      return off;
    }
    return -1;
  }
  void release(int64_t off, int64_t n) {
    if (n <= 0 || off < 0) return;
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t free_ranges() const { return free_.size(); }

 private:
  int64_t cap_ = 0, used_ = 0;
  std::map<int64_t, int64_t> free_;   // offset -> length, disjoint, not adjacent
};

// One request inside a batch.
template <class Request>
struct Item {
  uint64_t ticket = 0;
  Request req;
  int slot = -1;          // workspace of its lane
  int64_t cost = 0;       // arena units, set by phase A
  int64_t offset = -1;    // arena range granted by admission
  int status = 0;         // executor status (0 = ok)
  int64_t instances = 0;  // reported back to the caller
};

// The device side, called from the lane's own worker thread.  measure: phase A for the
// items of a batch on `lane` (their slots are assigned); returns once every item's cost (or
// an error status) is known.  launch: phase B for the admitted items.  finish: waits for the
// lane's launched work and sets each item's status and instance count.
template <class Request>
struct Executor {
  std::function<void(int lane, std::vector<Item<Request>>&)> measure;
  std::function<void(int lane, std::vector<Item<Request>>&)> launch;
  std::function<void(int lane, std::vector<Item<Request>>&)> finish;
};

enum class State { Pending, Measuring, Running, Done };

template <class Request>
struct Job {
  uint64_t ticket = 0;
  Request req;
  State state = State::Pending;
  int status = 0;
  int slot = -1;
  int64_t instances = 0;
  double t_submit = 0, t_start = 0, t_done = 0;   // seconds, steady clock
};

struct Result {
  int status;
  int slot;
  int64_t instances;
  double queue_us, run_us, latency_us;
};

template <class Request>
class Scheduler {
 public:
  static constexpr int kOk = 0, kBusy = 6, kOverBudget = 7, kArg = 1, kCancelled = 9;

  // lanes x slots_per_lane requests may be in flight; the arena has `arena_units` units;
  // a request that could not be admitted waits at most `aging_s` before it blocks the
  // requests behind it.
  Scheduler(int lanes, int slots_per_lane, int64_t arena_units, double aging_s, Executor<Request> ex)
      : spl_(slots_per_lane), aging_(aging_s), arena_(arena_units), ex_(std::move(ex)) {
    for (int l = 0; l < lanes; ++l) workers_.emplace_back([this, l] { work(l); });
  }

  ~Scheduler() { shutdown(); }

  void shutdown() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      if (stop_) return;
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : workers_)
      if (t.joinable()) t.join();
    std::lock_guard<std::mutex> lk(mu_);
    for (auto& kv : jobs_)
      if (kv.second.state == State::Pending) finish_locked(kv.second, kCancelled);
    pending_.clear();
    cv_done_.notify_all();
  }

  // Queue a request; `min_cost` is a lower bound of its arena need known without the GPU
  // (a request that can never fit is refused at once).
  int submit(const Request& r, int64_t min_cost, uint64_t* ticket) {
    if (!ticket || min_cost < 0) return kArg;
    std::lock_guard<std::mutex> lk(mu_);
    if (min_cost > arena_.capacity()) return kOverBudget;
    if (stop_) return kArg;
    Job<Request> j;
    j.ticket = ++next_ticket_;
    j.req = r;
    j.t_submit = now();
    jobs_[j.ticket] = j;
    pending_.push_back(j.ticket);
    *ticket = j.ticket;
    cv_.notify_all();
    return kOk;
  }

  // Wait up to timeout_us (0 = do not wait, < 0 = wait indefinitely) for a result.
  // kBusy if not finished in time; kArg for an unknown ticket.  A finished job's record
  // is released by the first poll that returns it.
  int poll(uint64_t ticket, int64_t timeout_us, Result* out) {
    std::unique_lock<std::mutex> lk(mu_);
    if (jobs_.find(ticket) == jobs_.end()) return kArg;
    auto done = [&] {
      auto it = jobs_.find(ticket);
      return it == jobs_.end() || it->second.state == State::Done;
    };
    if (!done()) {
      if (timeout_us == 0) return kBusy;
      if (timeout_us < 0)
        cv_done_.wait(lk, done);
      else if (!cv_done_.wait_for(lk, std::chrono::microseconds(timeout_us), done))
        return kBusy;
    }
    auto it = jobs_.find(ticket);
    if (it == jobs_.end()) return kArg;     // released by a concurrent poll
    const Job<Request>& j = it->second;
    if (out) {
      out->status = j.status;
      out->slot = j.slot;
      out->instances = j.instances;
      out->queue_us = 1e6 * ((j.t_start > 0 ? j.t_start : j.t_done) - j.t_submit);
      out->run_us = j.t_start > 0 ? 1e6 * (j.t_done - j.t_start) : 0.0;
      out->latency_us = 1e6 * (j.t_done - j.t_submit);
    }
    jobs_.erase(ticket);
    return kOk;
  }

  // Cancel a request that is waiting in the queue; kBusy once its batch has taken it.
  int cancel(uint64_t ticket) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = jobs_.find(ticket);
    if (it == jobs_.end()) return kArg;
    if (it->second.state != State::Pending) return kBusy;
    for (auto p = pending_.begin(); p != pending_.end(); ++p)
      if (*p == ticket) {
        pending_.erase(p);
        break;
      }
    finish_locked(it->second, kCancelled);
    cv_done_.notify_all();
    return kOk;
  }

  int64_t arena_used() {
    std::lock_guard<std::mutex> lk(mu_);
    return arena_.used();
  }
  int64_t arena_peak() {
    std::lock_guard<std::mutex> lk(mu_);
    return arena_peak_;
  }
  int64_t arena_capacity() {
    std::lock_guard<std::mutex> lk(mu_);
    return arena_.capacity();
  }
  int peak_running() {
    std::lock_guard<std::mutex> lk(mu_);
    return peak_running_;
  }
  int64_t batches() {
    std::lock_guard<std::mutex> lk(mu_);
    return batches_;
  }
  int peak_batch() {
    std::lock_guard<std::mutex> lk(mu_);
    return peak_batch_;
  }

 private:
  static double now() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
  }

  void finish_locked(Job<Request>& j, int status) {
    j.state = State::Done;
    j.status = status;
    j.t_done = now();
  }

  void work(int lane) {
    std::unique_lock<std::mutex> lk(mu_);
    uint64_t seen_release = 0;   // releases seen when this lane last admitted nothing
    bool waiting_memory = false;
    while (true) {
      cv_.wait(lk, [&] {
        return stop_ || (!pending_.empty() && (!waiting_memory || releases_ != seen_release));
      });
      if (stop_) return;
      waiting_memory = false;
      std::vector<Item<Request>> batch;
      while (!pending_.empty() && (int)batch.size() < spl_) {
        Job<Request>& j = jobs_[pending_.front()];
        pending_.pop_front();
        j.state = State::Measuring;
        Item<Request> it;
        it.ticket = j.ticket;
        it.req = j.req;
        it.slot = (int)batch.size();
        batch.push_back(it);
      }
      lk.unlock();
      ex_.measure(lane, batch);   // phase A: true costs
      lk.lock();
      std::vector<Item<Request>> admitted, back;
      bool hold = false;   // an aged request does not fit: admit nothing behind it
      for (Item<Request>& it : batch) {
        Job<Request>& j = jobs_[it.ticket];
        if (stop_) {
          finish_locked(j, kCancelled);
          continue;
        }
        if (hold) {
          back.push_back(it);
          continue;
        }
        if (it.status != kOk) {
          finish_locked(j, it.status);
          continue;
        }
        if (it.cost > arena_.capacity()) {
          finish_locked(j, kOverBudget);
          continue;
        }
        const int64_t off = arena_.alloc(it.cost);
        if (off >= 0) {
          it.offset = off;
          j.state = State::Running;
          j.t_start = now();
          admitted.push_back(it);
        } else {
          back.push_back(it);
          if (now() - j.t_submit > aging_) hold = true;
        }
      }
      for (auto r = back.rbegin(); r != back.rend(); ++r) {   // back to the head, in order
        jobs_[r->ticket].state = State::Pending;
        pending_.push_front(r->ticket);
      }
      if (arena_.used() > arena_peak_) arena_peak_ = arena_.used();
      cv_done_.notify_all();
      if (admitted.empty()) {
        // nothing fits until running requests free memory; if none is running the arena is
        // empty and every cost <= capacity was admitted, so this cannot stall
        waiting_memory = running_ > 0;
        seen_release = releases_;
        cv_.notify_all();
        continue;
      }
      running_ += (int)admitted.size();
      if (running_ > peak_running_) peak_running_ = running_;
      ++batches_;
      if ((int)admitted.size() > peak_batch_) peak_batch_ = (int)admitted.size();
      if (!back.empty()) cv_.notify_all();   // another lane may take what was put back
      lk.unlock();
      ex_.launch(lane, admitted);   // phase B
      ex_.finish(lane, admitted);   // wait for this lane's batch
      lk.lock();
      for (Item<Request>& it : admitted) {
        arena_.release(it.offset, it.cost);
        Job<Request>& j = jobs_[it.ticket];
        j.instances = it.instances;
        j.slot = lane * spl_ + it.slot;
        finish_locked(j, it.status);
      }
      running_ -= (int)admitted.size();
      ++releases_;
      cv_done_.notify_all();
      cv_.notify_all();
    }
  }

  const int spl_;
  const double aging_;
  Arena arena_;
  Executor<Request> ex_;
  std::mutex mu_;
  std::condition_variable cv_, cv_done_;
  std::deque<uint64_t> pending_;
  std::unordered_map<uint64_t, Job<Request>> jobs_;
  std::vector<std::thread> workers_;
  uint64_t next_ticket_ = 0, releases_ = 0;
  int64_t arena_peak_ = 0, batches_ = 0;
  int running_ = 0, peak_running_ = 0, peak_batch_ = 0;
  bool stop_ = false;
};

}  // namespace gs_serve
