"""Host-side logic of the serving scheduler (paper_2603_09632_gb300/csrc/serve_core.hpp),
driven by a fake executor on the CPU: continuous admission under the memory budget,
refusal of requests that can never fit, poll timeouts, cancellation of pending requests,
shutdown with requests still queued.  No GPU is involved."""
import ctypes as C
import os
import subprocess
import time

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OK, ARG, BUSY, OVER, CANCELLED = 0, 1, 6, 7, 9


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("serve") / "libserveharness.so")
    subprocess.run(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-pthread",
                    "-I" + os.path.join(ROOT, "paper_2603_09632_gb300", "csrc"),
                    os.path.join(HERE, "serve_harness.cpp"), "-o", out], check=True)
    L = C.CDLL(out)
    P, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    L.h_create.restype = P
    L.h_create.argtypes = [i32, i64]
    L.h_destroy.argtypes = [P]
    L.h_shutdown.argtypes = [P]
    L.h_submit.argtypes = [P, i64, i32, i64, C.POINTER(C.c_uint64)]
    L.h_poll.argtypes = [P, C.c_uint64, i64, C.POINTER(C.c_double)]
    L.h_cancel.argtypes = [P, C.c_uint64]
    L.h_peak_in_flight.restype = i64
    L.h_peak_in_flight.argtypes = [P]
    L.h_peak_running.argtypes = [P]
    L.h_executed.argtypes = [P]
    return L


def submit(H, h, sleep_us, cost, status=OK):
    t = C.c_uint64()
    s = H.h_submit(h, sleep_us, status, cost, C.byref(t))
    return s, t.value


def poll(H, h, t, timeout_us=-1):
    out = (C.c_double * 6)()
    s = H.h_poll(h, t, timeout_us, out)
    return s, list(out)


def test_requests_overlap_up_to_slots_and_budget(H):
    h = H.h_create(4, 1000)
    ts = [submit(H, h, 20_000, 300)[1] for _ in range(8)]
    res = [poll(H, h, t) for t in ts]
    assert all(s == OK and r[0] == OK for s, r in res)
    # 1000 / 300: at most 3 run at once although 4 slots exist
    assert H.h_peak_running(h) == 3
    assert H.h_peak_in_flight(h) == 900
    assert H.h_executed(h) == 8
    H.h_destroy(h)


def test_continuous_admission_beats_serial(H):
    h = H.h_create(4, 10_000)
    t0 = time.perf_counter()
    ts = [submit(H, h, 30_000, 100)[1] for _ in range(8)]
    for t in ts:
        assert poll(H, h, t)[0] == OK
    dt = time.perf_counter() - t0
    assert dt < 8 * 0.030 * 0.6           # 4 at a time: about two rounds, not eight
    H.h_destroy(h)


def test_request_larger_than_budget_is_refused(H):
    h = H.h_create(2, 1000)
    s, _ = submit(H, h, 1000, 1001)
    assert s == OVER
    s, _ = submit(H, h, 1000, -1)
    assert s == ARG
    H.h_destroy(h)


def test_poll_timeout_and_release(H):
    h = H.h_create(1, 1000)
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
    h = H.h_create(2, 1000)
    _, t1 = submit(H, h, 1000, 10, status=4)
    _, t2 = submit(H, h, 1000, 10, status=OK)
    assert poll(H, h, t1)[1][0] == 4
    assert poll(H, h, t2)[1][0] == OK
    H.h_destroy(h)


def test_cancel_pending_but_not_running(H):
    h = H.h_create(1, 1000)
    _, t1 = submit(H, h, 100_000, 10)
    time.sleep(0.02)                             # t1 is running now
    _, t2 = submit(H, h, 1000, 10)               # queued behind it
    assert H.h_cancel(h, t2) == OK
    assert H.h_cancel(h, t1) == BUSY
    s, r = poll(H, h, t2, 0)
    assert s == OK and r[0] == CANCELLED and r[1] == -1
    assert poll(H, h, t1)[1][0] == OK
    assert H.h_executed(h) == 1
    H.h_destroy(h)


def test_budget_blocks_until_memory_is_freed(H):
    h = H.h_create(2, 1000)
    _, big = submit(H, h, 80_000, 900)
    time.sleep(0.01)
    _, small = submit(H, h, 1000, 200)          # fits a slot but not the remaining budget
    assert poll(H, h, small, 20_000)[0] == BUSY
    s, r = poll(H, h, small, 2_000_000)
    assert s == OK and r[3] >= 50_000           # waited in the queue for the big one
    assert poll(H, h, big)[0] == OK
    H.h_destroy(h)


def test_shutdown_cancels_queued_requests(H):
    h = H.h_create(1, 1000)
    _, t1 = submit(H, h, 50_000, 10)
    time.sleep(0.01)
    ts = [submit(H, h, 50_000, 10)[1] for _ in range(3)]
    H.h_shutdown(h)
    assert poll(H, h, t1)[1][0] == OK
    assert all(poll(H, h, t, 0)[1][0] == CANCELLED for t in ts)
    H.h_destroy(h)
