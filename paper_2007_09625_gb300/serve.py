"""Continuous-batching request loop over the library's native server.

`Server` wraps gbsz_server_* (include/gbsz.h): requests arrive at any time
(`submit`), worker threads inside the library (each with its own context and
stream) take the oldest queued requests that fit the device-memory budget,
up to `max_batch` per batch, and run them with the batch entry points, so
batches of different workers overlap on the GPU.  A request's result is the
same bytes as a single-field call on the same input.  `stats()` reports p50 /
p99 latency and throughput, measured by the library.  This module only
allocates the output tensors and marshals pointers.
"""
import ctypes as C

import torch

from . import gbsz

COMPRESS, DECOMPRESS = "compress", "decompress"


class Request:
    __slots__ = ("srv", "ticket", "kind", "data", "out", "status", "error", "result", "out_bytes")

    def __init__(self, srv, ticket, kind, data, out):
        self.srv, self.ticket, self.kind, self.data, self.out = srv, ticket, kind, data, out
        self.status = None
        self.error = None
        self.result = None
        self.out_bytes = None

    def wait(self, timeout=None):
        """Blocks until done (or raises TimeoutError); returns (archive tensor,
        nbytes) for a compress, the field tensor for a decompress."""
        if self.error is not None:
            raise self.error
        if self.status is None:
            st = C.c_int()
            ob = C.c_size_t()
            r = gbsz.load().gbsz_server_wait(self.srv.h, C.c_uint64(self.ticket),
                                             C.c_double(-1.0 if timeout is None else float(timeout)),
                                             C.byref(st), C.byref(ob))
            if r == gbsz.ERR_TIMEOUT:
                raise TimeoutError(f"request {self.ticket} not done")
            if r != gbsz.OK:
                raise gbsz.GbszError(r, "gbsz_server_wait")
            self.status, self.out_bytes = st.value, ob.value
            self.result = (self.out, self.out_bytes) if self.kind == COMPRESS else self.out
        if self.status != gbsz.OK:
            raise gbsz.GbszError(self.status, f"request {self.ticket}")
        return self.result


class Server:
    def __init__(self, workers=2, max_batch=8, mem_budget=64 << 30, device=0):
        self.workers, self.max_batch, self.budget, self.device = workers, max_batch, mem_budget, device
        self.h = None

    def start(self):
        h = C.c_void_p()
        st = gbsz.load().gbsz_server_create(C.byref(h), self.device, self.workers, self.max_batch, int(self.budget))
        if st != gbsz.OK:
            raise gbsz.GbszError(st, "gbsz_server_create")
        self.h = h
        return self

    def submit(self, kind, data, nbytes=None, out=None, **params):
        """compress: data = contiguous float32 CUDA tensor, params eb, eb_mode,
        radius, chunk, lblock, order as for Context.compress.  decompress:
        data = uint8 CUDA archive tensor, nbytes its size.  The input must be
        complete on the device (the producing stream synchronised).  out: the
        output tensor (archive bytes, or the field), allocated here if None
        (an archive then gets the worst-case size)."""
        L = gbsz.load()
        t = C.c_uint64()
        if kind == COMPRESS:
            p = gbsz.make_params(gbsz.field_dims(data), params.get("eb", 1e-4), params.get("eb_mode", gbsz.EB_REL),
                                 params.get("radius", 512), params.get("chunk", 0), params.get("lblock", 0),
                                 params.get("order", 1))
            if out is None:
                out = torch.empty(L.gbsz_compress_bound(C.byref(p)), dtype=torch.uint8, device=data.device)
            assert out.dtype == torch.uint8 and out.is_contiguous()
            st = L.gbsz_server_submit_compress(self.h, C.c_void_p(data.data_ptr()), C.byref(p),
                                               C.c_void_p(out.data_ptr()), out.numel(), C.byref(t))
        else:
            nbytes = data.numel() if nbytes is None else int(nbytes)
            if out is None:
                p, n = gbsz.archive_info(data[:128].cpu().numpy(), nbytes)
                shape = [int(p.dims[i]) for i in range(p.ndim)][::-1]
                out = torch.empty(shape, dtype=torch.float32, device=data.device)
            assert out.dtype == torch.float32 and out.is_contiguous()
            st = L.gbsz_server_submit_decompress(self.h, C.c_void_p(data.data_ptr()), nbytes,
                                                 C.c_void_p(out.data_ptr()), out.numel(), C.byref(t))
        # the output's allocation is ordered on the current stream: let it
        # complete before a worker's stream writes the tensor
        torch.cuda.current_stream(data.device).synchronize()
        req = Request(self, t.value, kind, data, out)
        if st == gbsz.ERR_CAPACITY:
            req.status = "rejected"
            req.error = MemoryError(f"request needs more than the budget of {self.budget} bytes")
        elif st != gbsz.OK:
            raise gbsz.GbszError(st, "gbsz_server_submit")
        return req

    def stats(self):
        out = (C.c_double * 6)()
        st = gbsz.load().gbsz_server_stats(self.h, out)
        if st != gbsz.OK:
            raise gbsz.GbszError(st, "gbsz_server_stats")
        keys = ("requests", "p50_ms", "p99_ms", "mean_batch", "throughput_gbs", "span_s")
        d = dict(zip(keys, list(out)))
        d["requests"] = int(d["requests"])
        return d

    def memory(self):
        """Device memory the server counts against its budget: bytes now,
        their peak, scratch releases to admit requests, batches whose worker
        ended above its bound (0 unless the bound is wrong)."""
        out = (C.c_uint64 * 4)()
        st = gbsz.load().gbsz_server_memory(self.h, out)
        if st != gbsz.OK:
            raise gbsz.GbszError(st, "gbsz_server_memory")
        return dict(zip(("in_use", "peak", "releases", "overruns"), list(out)))

    def stop(self):
        if self.h:
            gbsz.load().gbsz_server_destroy(self.h)
            self.h = None
