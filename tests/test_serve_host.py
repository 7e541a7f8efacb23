"""Host logic of the continuous-batching loop, with a stand-in backend (no
GPU): admission by memory budget, batch size limit, admission of requests
that arrive while others run, rejection of requests above the budget."""
import threading
import time

import numpy as np

from paper_2007_09625_gb300.serve import COMPRESS, DECOMPRESS, Server


class FakeBackend:
    def __init__(self, delay=0.02):
        self.delay = delay
        self.lock = threading.Lock()
        self.running = 0
        self.max_running = 0
        self.max_mem = 0
        self.server = None

    def new_worker(self):
        return object()

    def memory_of(self, req):
        if req.kind == DECOMPRESS:
            req.params["shape"] = [int(req.nbytes)]
        return int(req.data.nbytes)

    def run(self, worker, reqs):
        with self.lock:
            self.running += len(reqs)
            self.max_running = max(self.max_running, self.running)
            self.max_mem = max(self.max_mem, self.server.in_use)
        time.sleep(self.delay)
        for r in reqs:
            r.result = r.data[::-1].copy()
            r.status = 0
        with self.lock:
            self.running -= len(reqs)


def test_all_requests_complete_within_limits():
    be = FakeBackend()
    srv = Server(backend=be, workers=3, max_batch=4, mem_budget=10_000)
    be.server = srv
    srv.start()
    rng = np.random.default_rng(0)
    reqs = []
    for i in range(40):
        data = rng.random(int(rng.integers(10, 300))).astype(np.float32)
        reqs.append(srv.submit(COMPRESS if i % 2 else DECOMPRESS, data, nbytes=data.size))
        time.sleep(0.002)
    for r in reqs:
        out = r.wait(10)
        assert np.array_equal(out, r.data[::-1])
    srv.stop()
    assert max(srv.batches) <= 4
    assert be.max_mem <= 10_000
    st = srv.stats()
    assert st["requests"] == 40 and st["p99_ms"] >= st["p50_ms"] > 0


def test_requests_arriving_during_work_are_admitted():
    be = FakeBackend(delay=0.2)
    srv = Server(backend=be, workers=2, max_batch=2, mem_budget=1 << 20)
    be.server = srv
    srv.start()
    first = srv.submit(COMPRESS, np.zeros(10, np.float32))
    time.sleep(0.05)  # the first batch is running now
    second = srv.submit(COMPRESS, np.ones(10, np.float32))
    second.wait(5)
    first.wait(5)
    srv.stop()
    # the second request started before the first finished: its work overlapped
    assert second.start < first.done_at
    assert be.max_running == 2


def test_memory_budget_serialises_and_rejects():
    be = FakeBackend(delay=0.05)
    srv = Server(backend=be, workers=4, max_batch=8, mem_budget=1000)
    be.server = srv
    srv.start()
    big = [srv.submit(COMPRESS, np.zeros(150, np.float32)) for _ in range(4)]  # 600 bytes each
    huge = srv.submit(COMPRESS, np.zeros(1000, np.float32))  # 4000 > budget
    for r in big:
        r.wait(5)
    assert huge.status == "rejected"
    srv.stop()
    assert be.max_mem <= 1000 and be.max_running == 1
