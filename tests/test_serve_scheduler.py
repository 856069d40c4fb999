"""Host-side logic of the serving scheduler (paper_2603_09632_gb300/csrc/serve_core.hpp),
driven by a fake executor on the CPU: batches of the oldest requests per free lane,
two-phase admission into a fixed arena by the cost phase A finds, refusal of requests that
can never fit, aging (a large request is not overtaken forever), poll timeouts,
cancellation of queued requests, shutdown with requests still queued, and the arena's
first-fit allocator.  No GPU is involved."""
import ctypes as C
import os
import subprocess
import threading
import time

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OK, ARG, DEVICE, BUSY, OVER, CANCELLED = 0, 1, 4, 6, 7, 9


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("serve") / "libserveharness.so")
    subprocess.run(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-pthread",
                    "-I" + os.path.join(ROOT, "paper_2603_09632_gb300", "csrc"),
                    os.path.join(HERE, "serve_harness.cpp"), "-o", out], check=True)
    L = C.CDLL(out)
    P, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    L.h_create.restype = P
    L.h_create.argtypes = [i32, i32, i64, C.c_double]
    L.h_destroy.argtypes = [P]
    L.h_shutdown.argtypes = [P]
    L.h_submit.argtypes = [P, i64, i32, i64, i64, i32, C.POINTER(C.c_uint64)]
    L.h_poll.argtypes = [P, C.c_uint64, i64, C.POINTER(C.c_double)]
    L.h_cancel.argtypes = [P, C.c_uint64]
    for f in ("h_arena_peak", "h_arena_used", "h_batches"):
        getattr(L, f).restype = i64
        getattr(L, f).argtypes = [P]
    for f in ("h_peak_running", "h_peak_batch", "h_executed", "h_measured"):
        getattr(L, f).argtypes = [P]
    L.h_arena_ops.restype = i64
    L.h_arena_ops.argtypes = [i64, i32, C.POINTER(i64), C.POINTER(i64)]
    return L


def create(H, lanes=2, spl=2, arena=1000, aging=0.05):
    return H.h_create(lanes, spl, arena, aging)


def submit(H, h, sleep_us, cost, status=OK, min_cost=0, measure_status=OK):
    t = C.c_uint64()
    s = H.h_submit(h, sleep_us, status, cost, min_cost, measure_status, C.byref(t))
    return s, t.value


def poll(H, h, t, timeout_us=-1):
    out = (C.c_double * 6)()
    s = H.h_poll(h, t, timeout_us, out)
    return s, list(out)


def test_requests_submitted_together_run_as_batches_within_the_arena(H):
    h = create(H, lanes=2, spl=2, arena=1000)
    ts = [submit(H, h, 20_000, 300)[1] for _ in range(8)]
    res = [poll(H, h, t) for t in ts]
    assert all(s == OK and r[0] == OK for s, r in res)
    assert all(r[2] == 300 for _, r in res)          # the cost phase A found
    # 1000 / 300: at most three requests hold arena ranges at once, although four fit
    # the lanes, and a batch holds up to two
    assert H.h_peak_running(h) == 3
    assert H.h_arena_peak(h) == 900
    assert H.h_peak_batch(h) == 2
    assert H.h_executed(h) == 8
    assert H.h_arena_used(h) == 0
    H.h_destroy(h)


def test_two_lanes_overlap_batches(H):
    h = create(H, lanes=2, spl=2, arena=10_000)
    t0 = time.perf_counter()
    ts = [submit(H, h, 30_000, 100)[1] for _ in range(8)]
    for t in ts:
        assert poll(H, h, t)[0] == OK
    dt = time.perf_counter() - t0
    assert dt < 8 * 0.030 * 0.6           # two batches of two at a time: about two rounds
    assert H.h_batches(h) <= 6
    H.h_destroy(h)


def test_refusals(H):
    h = create(H, arena=1000)
    assert submit(H, h, 1000, 10, min_cost=1001)[0] == OVER   # known too big at submit
    assert submit(H, h, 1000, 10, min_cost=-1)[0] == ARG
    s, t = submit(H, h, 1000, 1001)                          # found too big by phase A
    assert s == OK
    st, r = poll(H, h, t)
    assert st == OK and r[0] == OVER and r[1] == -1
    s, t = submit(H, h, 1000, 10, measure_status=DEVICE)     # phase A failed
    assert poll(H, h, t)[1][0] == DEVICE
    assert H.h_executed(h) == 0
    H.h_destroy(h)


def test_poll_timeout_and_release(H):
    h = create(H, lanes=1, spl=1)
    s, t = submit(H, h, 200_000, 10)
    assert s == OK
    assert poll(H, h, t, 0)[0] == BUSY          # not done, do not wait
    assert poll(H, h, t, 1000)[0] == BUSY       # 1 ms is not enough
    s, r = poll(H, h, t, 5_000_000)
    assert s == OK and r[0] == OK and r[5] >= 190_000
    assert poll(H, h, t, 0)[0] == ARG           # released by the first successful poll
    assert poll(H, h, 123456, 0)[0] == ARG      # unknown ticket
    H.h_destroy(h)


def test_executor_error_is_reported_per_request(H):
    h = create(H)
    _, t1 = submit(H, h, 1000, 10, status=DEVICE)
    _, t2 = submit(H, h, 1000, 10, status=OK)
    assert poll(H, h, t1)[1][0] == DEVICE
    assert poll(H, h, t2)[1][0] == OK
    H.h_destroy(h)


def test_cancel_queued_but_not_taken(H):
    h = create(H, lanes=1, spl=1)
    _, t1 = submit(H, h, 100_000, 10)
    time.sleep(0.02)                             # t1 is on the device now
    _, t2 = submit(H, h, 1000, 10)               # queued behind it
    assert H.h_cancel(h, t2) == OK
    assert H.h_cancel(h, t1) == BUSY
    s, r = poll(H, h, t2, 0)
    assert s == OK and r[0] == CANCELLED and r[1] == -1
    assert poll(H, h, t1)[1][0] == OK
    assert H.h_executed(h) == 1
    H.h_destroy(h)


def test_admission_waits_until_memory_is_freed(H):
    h = create(H, lanes=2, spl=1, arena=1000)
    _, big = submit(H, h, 80_000, 900)
    time.sleep(0.01)
    _, small = submit(H, h, 1000, 200)          # a lane is free but the arena is not
    assert poll(H, h, small, 20_000)[0] == BUSY
    s, r = poll(H, h, small, 2_000_000)
    assert s == OK and r[3] >= 50_000           # waited in the queue for the big one
    assert poll(H, h, big)[0] == OK
    assert H.h_measured(h) >= 3                 # the small one was measured again
    H.h_destroy(h)


def test_large_request_is_not_overtaken_forever(H):
    """Small requests keep arriving and each would fit beside the others; a large request
    that needs most of the arena is admitted once it has waited past the aging limit,
    because nothing behind it is admitted from then on."""
    h = create(H, lanes=2, spl=2, arena=1000, aging=0.02)
    stop = threading.Event()
    smalls = []

    def feeder():
        while not stop.is_set():
            smalls.append(submit(H, h, 5_000, 300)[1])
            time.sleep(0.002)

    th = threading.Thread(target=feeder)
    th.start()
    time.sleep(0.02)
    _, big = submit(H, h, 5_000, 800)
    s, r = poll(H, h, big, 2_000_000)
    stop.set()
    th.join()
    assert s == OK and r[0] == OK
    assert r[3] < 500_000                        # admitted well within the run
    for t in smalls:
        assert poll(H, h, t, 5_000_000)[0] == OK
    H.h_destroy(h)


def test_shutdown_cancels_queued_requests(H):
    h = create(H, lanes=1, spl=1)
    _, t1 = submit(H, h, 50_000, 10)
    time.sleep(0.01)
    ts = [submit(H, h, 50_000, 10)[1] for _ in range(3)]
    H.h_shutdown(h)
    assert poll(H, h, t1)[1][0] == OK
    assert all(poll(H, h, t, 0)[1][0] == CANCELLED for t in ts)
    H.h_destroy(h)


def test_arena_first_fit_and_coalescing(H):
    def run(cap, ops):
        n = len(ops)
        op = (C.c_int64 * n)(*ops)
        res = (C.c_int64 * n)()
        free_ranges = H.h_arena_ops(cap, n, op, res)
        return list(res), free_ranges

    # three ranges, release the middle, a request that fits the hole takes it
    res, fr = run(100, [30, 30, 30, -2, 20])
    assert res[:3] == [0, 30, 60] and res[4] == 30
    # too big for any free range, although enough units are free in total
    res, fr = run(100, [40, 20, 40, -1, -3, 50])
    assert res[:3] == [0, 40, 60] and res[5] == -1
    # releasing everything merges the ranges back into one
    res, fr = run(100, [10, 20, 30, -2, -1, -3])
    assert fr == 1 and res[-1] == 0
