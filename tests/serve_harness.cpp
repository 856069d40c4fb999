// Test harness: the serving scheduler (serve_core.hpp) driven by a fake executor, so the
// host-side logic (batching, two-phase admission into the arena, queueing, aging, poll
// timeouts, cancellation, shutdown) is tested on the CPU without a GPU.  Phase A of the
// fake reports each request's declared cost (or its declared phase-A error); a batch
// "runs" from its launch until its longest request's duration has passed, and each request
// then finishes with the status it asks for.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <thread>

#include "serve_core.hpp"

namespace {

struct FakeReq {
  int64_t sleep_us;
  int status;        // final status
  int64_t cost;      // arena units found by phase A
  int measure_status;
};

using Item = gs_serve::Item<FakeReq>;

struct Harness {
  std::atomic<int> executed{0}, measured{0};
  std::chrono::steady_clock::time_point t_launch[4];
  int64_t batch_us[4] = {0, 0, 0, 0};
  gs_serve::Scheduler<FakeReq>* sched = nullptr;
};

}  // namespace

extern "C" {

void* h_create(int lanes, int slots_per_lane, int64_t arena, double aging_s) {
  Harness* h = new Harness();
  gs_serve::Executor<FakeReq> ex;
  ex.measure = [h](int, std::vector<Item>& b) {
    for (Item& it : b) {
      it.cost = it.req.cost;
      it.status = it.req.measure_status;
      h->measured.fetch_add(1);
    }
  };
  ex.launch = [h](int lane, std::vector<Item>& b) {
    h->t_launch[lane] = std::chrono::steady_clock::now();
    int64_t us = 0;
    for (Item& it : b) us = std::max(us, it.req.sleep_us);
    h->batch_us[lane] = us;
  };
  ex.finish = [h](int lane, std::vector<Item>& b) {
    std::this_thread::sleep_until(h->t_launch[lane] + std::chrono::microseconds(h->batch_us[lane]));
    for (Item& it : b) {
      it.status = it.req.status;
      it.instances = it.cost;
      h->executed.fetch_add(1);
    }
  };
  h->sched = new gs_serve::Scheduler<FakeReq>(lanes, slots_per_lane, arena, aging_s, ex);
  return h;
}

void h_destroy(void* p) {
  Harness* h = static_cast<Harness*>(p);
  delete h->sched;
  delete h;
}

void h_shutdown(void* p) { static_cast<Harness*>(p)->sched->shutdown(); }

int h_submit(void* p, int64_t sleep_us, int status, int64_t cost, int64_t min_cost,
             int measure_status, uint64_t* ticket) {
  return static_cast<Harness*>(p)->sched->submit(FakeReq{sleep_us, status, cost, measure_status},
                                                 min_cost, ticket);
}

// out: status, slot, instances, queue_us, run_us, latency_us
int h_poll(void* p, uint64_t ticket, int64_t timeout_us, double* out) {
  gs_serve::Result r;
  const int s = static_cast<Harness*>(p)->sched->poll(ticket, timeout_us, &r);
  if (s == 0 && out) {
    out[0] = r.status;
    out[1] = r.slot;
    out[2] = (double)r.instances;
    out[3] = r.queue_us;
    out[4] = r.run_us;
    out[5] = r.latency_us;
  }
  return s;
}

int h_cancel(void* p, uint64_t ticket) { return static_cast<Harness*>(p)->sched->cancel(ticket); }

int64_t h_arena_peak(void* p) { return static_cast<Harness*>(p)->sched->arena_peak(); }
int64_t h_arena_used(void* p) { return static_cast<Harness*>(p)->sched->arena_used(); }
int h_peak_running(void* p) { return static_cast<Harness*>(p)->sched->peak_running(); }
int h_peak_batch(void* p) { return static_cast<Harness*>(p)->sched->peak_batch(); }
int64_t h_batches(void* p) { return static_cast<Harness*>(p)->sched->batches(); }
int h_executed(void* p) { return static_cast<Harness*>(p)->executed.load(); }
int h_measured(void* p) { return static_cast<Harness*>(p)->measured.load(); }

// Arena allocator alone: n operations (op[k] > 0: allocate op[k] units, result in res[k];
// op[k] < 0: release the range allocated by operation -op[k] - 1).  Returns the number of
// free ranges left.
int64_t h_arena_ops(int64_t cap, int n, const int64_t* op, int64_t* res) {
  gs_serve::Arena a(cap);
  for (int k = 0; k < n; ++k) {
    if (op[k] > 0) {
      res[k] = a.alloc(op[k]);
    } else {
      const int j = (int)(-op[k] - 1);
      a.release(res[j], op[j]);
      res[k] = a.used();
    }
  }
  return (int64_t)a.free_ranges();
}

}  // extern "C"
