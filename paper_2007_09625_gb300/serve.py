"""Continuous-batching request loop for compress / decompress requests.

Requests arrive at any time (`submit`).  Worker threads, each with its own
library context and CUDA stream, repeatedly take the oldest queued requests
that fit the device-memory budget (up to `max_batch` per batch) and run them
with the library's batch entry points, whose fields run concurrently on
several streams.  A request that arrives while others are on the GPU is
admitted as soon as a worker is free and memory allows, so the work of
several batches overlaps on the device.  Each request records its arrival,
start and completion times; `stats()` reports p50 / p99 latency and
throughput.  Results are independent of batching: a request's output is the
same bytes as a single-field call on the same input.

The backend is the CUDA library through `gbsz`; tests of the host logic pass
a stand-in backend with the same three methods.
"""
import collections
import threading
import time

import numpy as np

COMPRESS, DECOMPRESS = "compress", "decompress"


def _numel(x):
    return x.numel() if hasattr(x, "numel") else int(np.size(x))


class Request:
    __slots__ = ("id", "kind", "data", "nbytes", "params", "mem", "arrival", "start", "done_at", "result",
                 "status", "error", "event")

    def __init__(self, rid, kind, data, params=None, nbytes=None):
        self.id = rid
        self.kind = kind
        self.data = data        # compress: float32 field tensor; decompress: uint8 archive tensor
        self.nbytes = nbytes    # decompress: archive bytes
        self.params = params or {}
        self.mem = 0
        self.arrival = time.perf_counter()
        self.start = self.done_at = None
        self.result = None      # compress: (archive tensor, nbytes); decompress: field tensor
        self.status = None
        self.error = None
        self.event = threading.Event()

    def wait(self, timeout=None):
        if not self.event.wait(timeout):
            raise TimeoutError(f"request {self.id} not done")
        if self.error is not None:
            raise self.error
        return self.result


class CudaBackend:
    """The library through its Python binding: one context per worker."""

    def __init__(self, device=0):
        from . import gbsz
        self.gbsz = gbsz
        self.device = device

    def new_worker(self):
        import torch
        ctx = self.gbsz.Context(self.device)
        stream = torch.cuda.Stream(device=self.device)
        return ctx, stream

    def memory_of(self, req):
        """Device bytes a request needs while it runs: its output plus the
        context scratch that grows with the field (codes, residuals)."""
        if req.kind == COMPRESS:
            n = req.data.numel()
            p = req.params
            bound = self.gbsz.compress_bound(self.gbsz.field_dims(req.data), p.get("eb", 1e-4),
                                             p.get("eb_mode", 1), p.get("radius", 512), p.get("chunk", 0))
            return bound + 10 * n
        hdr = req.data[:128].cpu().numpy()
        p, n = self.gbsz.archive_info(hdr, req.nbytes)
        req.params["shape"] = [int(p.dims[i]) for i in range(p.ndim)][::-1]
        return 14 * n

    def run(self, worker, reqs):
        import torch
        ctx, stream = worker
        comp = [r for r in reqs if r.kind == COMPRESS]
        dec = [r for r in reqs if r.kind == DECOMPRESS]
        with torch.cuda.stream(stream):
            if comp:
                ps = [self.gbsz.make_params(self.gbsz.field_dims(r.data), r.params.get("eb", 1e-4),
                                            r.params.get("eb_mode", 1), r.params.get("radius", 512),
                                            r.params.get("chunk", 0)) for r in comp]
                try:
                    outs, nbs, sts = ctx.compress_batch([r.data for r in comp], None, params=ps, stream=stream)
                except self.gbsz.GbszError as e:
                    for r in comp:
                        r.error = e
                    outs, nbs, sts = [None] * len(comp), [0] * len(comp), [e.status] * len(comp)
                for r, o, nb, st in zip(comp, outs, nbs, sts):
                    r.result, r.status = (o, nb), st
            if dec:
                outs = [torch.empty(r.params["shape"], dtype=torch.float32, device=r.data.device) for r in dec]
                try:
                    outs, sts = ctx.decompress_batch([r.data for r in dec], [r.nbytes for r in dec], outs,
                                                     stream=stream)
                except self.gbsz.GbszError as e:
                    for r in dec:
                        r.error = e
                    sts = [e.status] * len(dec)
                for r, o, st in zip(dec, outs, sts):
                    r.result, r.status = o, st
        stream.synchronize()


class Server:
    def __init__(self, backend=None, workers=2, max_batch=8, mem_budget=64 << 30):
        self.backend = backend if backend is not None else CudaBackend()
        self.nworkers = workers
        self.max_batch = max_batch
        self.budget = mem_budget
        self.in_use = 0
        self.queue = collections.deque()
        self.cv = threading.Condition()
        self.stop_flag = False
        self.threads = []
        self.done = []
        self.next_id = 0
        self.batches = []  # sizes of the batches that ran

    # -- client side -------------------------------------------------------
    def submit(self, kind, data, nbytes=None, **params):
        with self.cv:
            req = Request(self.next_id, kind, data, dict(params), nbytes)
            self.next_id += 1
        req.mem = self.backend.memory_of(req)
        with self.cv:
            if req.mem > self.budget:
                req.status = "rejected"
                req.error = MemoryError(f"request {req.id} needs {req.mem} bytes, budget {self.budget}")
                req.event.set()
                return req
            self.queue.append(req)
            self.cv.notify()
        return req

    def start(self):
        for _ in range(self.nworkers):
            t = threading.Thread(target=self._worker, daemon=True)
            t.start()
            self.threads.append(t)
        return self

    def stop(self):
        with self.cv:
            self.stop_flag = True
            self.cv.notify_all()
        for t in self.threads:
            t.join()
        self.threads = []

    # -- scheduling --------------------------------------------------------
    def _take_batch(self):
        """Oldest requests first, as many as fit the budget and max_batch."""
        with self.cv:
            while True:
                if self.stop_flag and not self.queue:
                    return None
                batch = []
                while self.queue and len(batch) < self.max_batch:
                    r = self.queue[0]
                    if self.in_use + r.mem > self.budget:
                        break
                    self.queue.popleft()
                    self.in_use += r.mem
                    batch.append(r)
                if batch:
                    return batch
                self.cv.wait(0.05)

    def _release(self, batch):
        with self.cv:
            for r in batch:
                self.in_use -= r.mem
            self.cv.notify_all()

    def _worker(self):
        worker = self.backend.new_worker()
        while True:
            batch = self._take_batch()
            if batch is None:
                return
            t0 = time.perf_counter()
            for r in batch:
                r.start = t0
            try:
                self.backend.run(worker, batch)
            except Exception as e:  # pragma: no cover - surfaced to every request
                for r in batch:
                    r.error = e
            t1 = time.perf_counter()
            self._release(batch)
            with self.cv:
                self.batches.append(len(batch))
                for r in batch:
                    r.done_at = t1
                    self.done.append(r)
            for r in batch:
                r.event.set()

    # -- metrics -------------------------------------------------------------
    def stats(self):
        with self.cv:
            done = [r for r in self.done if r.error is None]
        if not done:
            return {}
        lat = np.array([r.done_at - r.arrival for r in done])
        t0 = min(r.arrival for r in done)
        t1 = max(r.done_at for r in done)
        in_bytes = sum(4 * _numel(r.data) if r.kind == COMPRESS else 4 * int(np.prod(r.params["shape"]))
                       for r in done)
        return {"requests": len(done), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_batch": float(np.mean(self.batches)),
                "throughput_gbs": in_bytes / (t1 - t0) / 1e9, "span_s": t1 - t0}
