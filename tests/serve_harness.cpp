// Test harness: the serving scheduler (serve_core.hpp) driven by a fake executor, so the
// host-side logic (admission by budget, queueing, poll timeouts, cancellation, shutdown)
// is tested on the CPU without a GPU.  The fake "runs" a request by sleeping for its
// duration and returns the status the request asks for.
#include <atomic>
#include <chrono>
#include <thread>

#include "serve_core.hpp"

namespace {

struct FakeReq {
  int64_t sleep_us;
  int status;
};

struct Harness {
  std::atomic<int> executed{0};
  gs_serve::Scheduler<FakeReq>* sched = nullptr;
};

}  // namespace

extern "C" {

void* h_create(int slots, int64_t budget) {
  Harness* h = new Harness();
  h->sched = new gs_serve::Scheduler<FakeReq>(slots, budget, [h](int, const FakeReq& r, int64_t* inst) {
    std::this_thread::sleep_for(std::chrono::microseconds(r.sleep_us));
    *inst = r.sleep_us;
    h->executed.fetch_add(1);
    return r.status;
  });
  return h;
}

void h_destroy(void* p) {
  Harness* h = static_cast<Harness*>(p);
  delete h->sched;
  delete h;
}

void h_shutdown(void* p) { static_cast<Harness*>(p)->sched->shutdown(); }

int h_submit(void* p, int64_t sleep_us, int status, int64_t cost, uint64_t* ticket) {
  return static_cast<Harness*>(p)->sched->submit(FakeReq{sleep_us, status}, cost, ticket);
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

int64_t h_peak_in_flight(void* p) { return static_cast<Harness*>(p)->sched->peak_in_flight_bytes(); }
int h_peak_running(void* p) { return static_cast<Harness*>(p)->sched->peak_running(); }
int h_executed(void* p) { return static_cast<Harness*>(p)->executed.load(); }

}  // extern "C"
