// Host-side scheduler of the serving loop (pure C++; no CUDA here, so its admission,
// queueing, timeout and cancellation logic can be exercised without a GPU).
//
// Requests are admitted continuously: a worker per slot takes the oldest pending request
// whose memory estimate fits the remaining budget, runs it through the executor and
// publishes the result; requests that arrive while others are running start as soon as
// a slot and enough budget are free, so their device work overlaps with the running ones.
#pragma once

#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <functional>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace gs_serve {

enum class State { Pending, Running, Done };

template <class Request>
struct Job {
  uint64_t ticket = 0;
  Request req;
  int64_t cost = 0;            // admission estimate (bytes)
  State state = State::Pending;
  int status = 0;              // executor status (0 = ok)
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

// Executor: runs one request on slot `slot`; returns a status (0 = ok) and the instance
// count through `instances`.
template <class Request>
using Executor = std::function<int(int slot, const Request&, int64_t* instances)>;

template <class Request>
class Scheduler {
 public:
  static constexpr int kOk = 0, kBusy = 6, kOverBudget = 7, kArg = 1, kCancelled = 9;

  Scheduler(int n_slots, int64_t budget, Executor<Request> exec)
      : budget_(budget), exec_(std::move(exec)) {
    for (int s = 0; s < n_slots; ++s) workers_.emplace_back([this, s] { work(s); });
  }

  ~Scheduler() { shutdown(); }

  void shutdown() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      if (stop_) return;
      stop_ = true;
    }
    cv_work_.notify_all();
    for (auto& t : workers_)
      if (t.joinable()) t.join();
    // requests still pending are cancelled
    std::lock_guard<std::mutex> lk(mu_);
    for (auto& kv : jobs_)
      if (kv.second.state == State::Pending) finish_locked(kv.second, kCancelled);
    pending_.clear();
    cv_done_.notify_all();
  }

  // Queue a request whose device memory estimate is `cost` bytes.  A request that could
  // never fit the budget is refused at once.
  int submit(const Request& r, int64_t cost, uint64_t* ticket) {
    if (!ticket || cost < 0) return kArg;
    std::lock_guard<std::mutex> lk(mu_);
    if (cost > budget_) return kOverBudget;
    if (stop_) return kArg;
    Job<Request> j;
    j.ticket = ++next_ticket_;
    j.req = r;
    j.cost = cost;
    j.t_submit = now();
    jobs_[j.ticket] = j;
    pending_.push_back(j.ticket);
    *ticket = j.ticket;
    cv_work_.notify_one();
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

  // Cancel a request that has not started; kBusy if it is already running or done.
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

  // Change the budget available to requests (e.g. after resident data took a share).
  void set_budget(int64_t b) {
    {
      std::lock_guard<std::mutex> lk(mu_);
      budget_ = b;
    }
    cv_work_.notify_all();
  }

  int64_t in_flight_bytes() {
    std::lock_guard<std::mutex> lk(mu_);
    return in_flight_;
  }
  int64_t peak_in_flight_bytes() {
    std::lock_guard<std::mutex> lk(mu_);
    return peak_in_flight_;
  }
  int peak_running() {
    std::lock_guard<std::mutex> lk(mu_);
    return peak_running_;
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

  // Oldest pending request that fits the remaining budget (FIFO among those that fit).
  bool take_locked(uint64_t* ticket) {
    for (auto p = pending_.begin(); p != pending_.end(); ++p) {
      Job<Request>& j = jobs_[*p];
      if (in_flight_ + j.cost <= budget_) {
        *ticket = *p;
        pending_.erase(p);
        return true;
      }
    }
    return false;
  }

  void work(int slot) {
    std::unique_lock<std::mutex> lk(mu_);
    while (true) {
      uint64_t t = 0;
      cv_work_.wait(lk, [&] { return stop_ || take_locked(&t); });
      if (stop_ && t == 0) return;
      Job<Request>& j = jobs_[t];
      j.state = State::Running;
      j.slot = slot;
      j.t_start = now();
      in_flight_ += j.cost;
      if (in_flight_ > peak_in_flight_) peak_in_flight_ = in_flight_;
      ++running_;
      if (running_ > peak_running_) peak_running_ = running_;
      const Request req = j.req;
      lk.unlock();
      int64_t inst = 0;
      const int st = exec_(slot, req, &inst);
      lk.lock();
      Job<Request>& jd = jobs_[t];
      jd.instances = inst;
      finish_locked(jd, st);
      in_flight_ -= jd.cost;
      --running_;
      cv_done_.notify_all();
      cv_work_.notify_all();   // budget freed: another waiting request may fit now
    }
  }

  int64_t budget_;
  Executor<Request> exec_;
  std::mutex mu_;
  std::condition_variable cv_work_, cv_done_;
  std::deque<uint64_t> pending_;
  std::unordered_map<uint64_t, Job<Request>> jobs_;
  std::vector<std::thread> workers_;
  uint64_t next_ticket_ = 0;
  int64_t in_flight_ = 0, peak_in_flight_ = 0;
  int running_ = 0, peak_running_ = 0;
  bool stop_ = false;
};

}  // namespace gs_serve
