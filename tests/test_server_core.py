"""Host logic of the native serving loop (server_core.h) with a stand-in
executor, no GPU: FIFO admission by a device-memory budget that counts every
worker's resident memory (idle or busy), release of a worker's scratch when
it blocks admission, batch size limit, admission of requests that arrive
while others run, rejection of requests above the budget, tickets and
latency statistics.  The harness is compiled here with the host compiler."""
import ctypes as C
import os
import subprocess
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "server_core_harness.cpp")
INC = os.path.join(ROOT, "paper_2007_09625_gb300", "csrc")
LIB = os.path.join(ROOT, "_build", "libserver_core_harness.so")


@pytest.fixture(scope="module")
def lib():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    hdr = os.path.join(INC, "server_core.h")
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(hdr)):
        subprocess.run(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread", "-I" + INC, SRC, "-o", LIB],
                       check=True)
    L = C.CDLL(LIB)
    P, u32, u64 = C.c_void_p, C.c_uint32, C.c_uint64
    L.h_new.argtypes, L.h_new.restype = [u32, u32, u64, C.c_int, u64], P
    L.h_submit.argtypes, L.h_submit.restype = [P, C.c_int, u64, u64], u64
    L.h_wait.argtypes, L.h_wait.restype = [P, u64, C.c_double, C.POINTER(C.c_int), C.POINTER(u64)], C.c_int
    L.h_poll.argtypes, L.h_poll.restype = [P, u64, C.POINTER(C.c_int), C.POINTER(u64)], C.c_int
    L.h_stats.argtypes = [P, P]
    L.h_times.argtypes = [P, u64, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.h_limits.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(u64)]
    L.h_memory.argtypes = [P] + [C.POINTER(u64)] * 4
    L.h_stop.argtypes = [P]
    L.h_free.argtypes = [P]
    return L


def wait(L, h, t, timeout=10.0):
    st, ob = C.c_int(), C.c_uint64()
    assert L.h_wait(h, t, timeout, C.byref(st), C.byref(ob)) == 1
    return st.value, ob.value


def limits(L, h):
    a, b, m = C.c_int(), C.c_int(), C.c_uint64()
    L.h_limits(h, C.byref(a), C.byref(b), C.byref(m))
    return a.value, b.value, m.value


def stats(L, h):
    out = (C.c_double * 6)()
    L.h_stats(h, out)
    return list(out)


def test_all_requests_complete_within_limits(lib):
    h = lib.h_new(3, 4, 10_000, 20, 0)
    tickets = []
    for i in range(40):
        n = 10 + (i * 37) % 290
        tickets.append((lib.h_submit(h, i % 2, n, 4 * n), n, i % 2))
        time.sleep(0.002)
    for t, n, k in tickets:
        assert t > 0
        assert wait(lib, h, t) == (0, 2 * n + k)
    # a ticket is released once its result was read
    st, ob = C.c_int(), C.c_uint64()
    assert lib.h_poll(h, tickets[0][0], C.byref(st), C.byref(ob)) == -1
    lib.h_stop(h)
    running, batch, mem = limits(lib, h)
    assert batch <= 4 and mem <= 10_000
    s = stats(lib, h)
    assert s[0] == 40 and s[2] >= s[1] > 0 and 1 <= s[3] <= 4
    lib.h_free(h)


def test_requests_arriving_during_work_are_admitted(lib):
    h = lib.h_new(2, 2, 1 << 20, 200, 0)
    first = lib.h_submit(h, 0, 10, 40)
    time.sleep(0.05)  # the first batch is running now
    second = lib.h_submit(h, 0, 10, 40)
    wait(lib, h, second)
    wait(lib, h, first)
    lib.h_stop(h)
    t0a, t1a, t0b, t1b = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    lib.h_times(h, first, C.byref(t0a), C.byref(t1a))
    lib.h_times(h, second, C.byref(t0b), C.byref(t1b))
    assert t0b.value < t1a.value  # the second started before the first finished
    assert limits(lib, h)[0] == 2
    lib.h_free(h)


def test_memory_budget_serialises_and_rejects(lib):
    h = lib.h_new(4, 8, 1000, 50, 0)
    big = [lib.h_submit(h, 0, 150, 600) for _ in range(4)]  # 600 bytes each: one at a time
    assert lib.h_submit(h, 0, 1000, 4000) == 0  # above the whole budget: rejected
    for t in big:
        wait(lib, h, t)
    lib.h_stop(h)
    running, batch, mem = limits(lib, h)
    assert mem <= 1000 and running == 1
    lib.h_free(h)


def test_poll_pending_then_done_and_stop_drains(lib):
    h = lib.h_new(1, 1, 1 << 20, 100, 0)
    ts = [lib.h_submit(h, 1, 5, 1) for _ in range(3)]
    st, ob = C.c_int(), C.c_uint64()
    assert lib.h_poll(h, ts[2], C.byref(st), C.byref(ob)) == 0  # queued behind the others
    st_, ob_ = C.c_int(), C.c_uint64()
    assert lib.h_wait(h, ts[2], 0.01, C.byref(st_), C.byref(ob_)) == 0  # timed out, still pending
    lib.h_stop(h)  # runs everything queued
    assert lib.h_submit(h, 0, 5, 1) == 0  # no new work after stop
    assert stats(lib, h)[0] == 3
    lib.h_free(h)


def memory(L, h):
    v = [C.c_uint64() for _ in range(4)]
    L.h_memory(h, *[C.byref(x) for x in v])
    return [x.value for x in v]


def test_resident_memory_counts_against_the_budget(lib):
    """Each worker holds 100 bytes of fixed tables plus the scratch of the
    largest request it ran; idle workers' memory stays counted, and a worker
    whose memory blocks the next request releases it."""
    h = lib.h_new(3, 4, 2000, 30, 100)
    assert memory(lib, h)[0] == 300  # three idle workers, fixed tables only
    ts = [lib.h_submit(h, i % 2, 100, 900) for i in range(6)]  # 900-byte scratch: one at a time
    assert lib.h_submit(h, 0, 10, 1901) == 0  # above the budget with one worker's tables
    for t in ts:
        assert wait(lib, h, t)[0] == 0
    lib.h_stop(h)
    in_use, peak, trims, over = memory(lib, h)
    assert peak <= 2000 and over == 0
    assert trims >= 1  # a worker holding 1000 bytes had to let go for another to run
    assert limits(lib, h)[2] <= 2000
    lib.h_free(h)


def test_small_requests_share_the_budget(lib):
    h = lib.h_new(4, 8, 10_000, 10, 100)
    ts = [lib.h_submit(h, 0, 10, 50 + i) for i in range(64)]
    for t in ts:
        assert wait(lib, h, t)[0] == 0
    lib.h_stop(h)
    in_use, peak, trims, over = memory(lib, h)
    assert peak <= 10_000 and over == 0 and trims == 0
    s = stats(lib, h)
    assert s[0] == 64 and s[3] > 1  # batched
    lib.h_free(h)
