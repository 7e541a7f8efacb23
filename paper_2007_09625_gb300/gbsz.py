"""Python binding of the C ABI in include/gbsz.h (argument marshalling only).

Every step of compression and decompression runs in the CUDA kernels of
libgbsz.so; this module only passes torch device pointers, sizes and the
current CUDA stream.  There is no CPU fallback: if the library is missing
or cannot load, every call raises.
"""
import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# GBSZ_LIBRARY: another build of the library (the bounds-checking one)
LIB_PATH = os.environ.get("GBSZ_LIBRARY") or os.path.join(_HERE, "libgbsz.so")

OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_CORRUPT, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_BOUNDS = range(9)
EB_ABS, EB_REL = 0, 1
NSTAGE = 11
STAGES = ["error_bound", "dualquant_hist", "codebook", "encode_count", "encode_scan", "encode_pack",
          "decode_tables", "decode_offsets", "decode", "reconstruct", "other"]
DEBUG_CODES, DEBUG_HIST, DEBUG_SCALARS, DEBUG_DECODED, DEBUG_CODEWORDS, DEBUG_GRAPHS, DEBUG_GRAPHS_SINGLE = range(7)

# every entry point of include/gbsz.h with its ctypes signature
_P = C.c_void_p
SIGNATURES = {
    "gbsz_create": ([C.POINTER(C.c_void_p), C.c_int], C.c_int),
    "gbsz_destroy": ([_P], None),
    "gbsz_compress_bound": ([_P], C.c_size_t),
    "gbsz_auto_chunk": ([_P], C.c_uint32),
    "gbsz_compress": ([_P, _P, _P, _P, C.c_size_t, C.POINTER(C.c_size_t), _P], C.c_int),
    "gbsz_decompress": ([_P, _P, C.c_size_t, _P, C.c_uint64, _P], C.c_int),
    "gbsz_compress_host": ([_P, _P, _P, _P, C.c_size_t, C.POINTER(C.c_size_t), _P], C.c_int),
    "gbsz_decompress_host": ([_P, _P, C.c_size_t, _P, C.c_uint64, _P], C.c_int),
    "gbsz_archive_info": ([_P, C.c_size_t, _P, C.POINTER(C.c_uint64)], C.c_int),
    "gbsz_status_str": ([C.c_int], C.c_char_p),
    "gbsz_debug_copy": ([_P, C.c_int, _P, C.c_size_t], C.c_int),
    "gbsz_profile_enable": ([_P, C.c_int], C.c_int),
    "gbsz_profile_read": ([_P, _P, _P, C.POINTER(C.c_uint64)], C.c_int),
    "gbsz_codebook_noalloc": ([_P, C.c_uint32, _P, _P, C.POINTER(C.c_uint32), _P], C.c_int),
    "gbsz_compress_batch": ([_P, C.c_uint32, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "gbsz_decompress_batch": ([_P, C.c_uint32, _P, _P, _P, _P, _P, _P], C.c_int),
    "gbsz_autotune": ([_P, _P, _P, _P, C.POINTER(C.c_float), _P], C.c_int),
    "gbsz_set_option": ([_P, C.c_int, C.c_int64], C.c_int),
    "gbsz_decompress_host_async": ([_P, _P, C.c_size_t, _P, C.c_uint64, _P], C.c_int),
    "gbsz_async_wait": ([_P], C.c_int),
    "gbsz_server_create": ([C.POINTER(C.c_void_p), C.c_int, C.c_uint32, C.c_uint32, C.c_uint64], C.c_int),
    "gbsz_server_destroy": ([_P], None),
    "gbsz_server_submit_compress": ([_P, _P, _P, _P, C.c_size_t, C.POINTER(C.c_uint64)], C.c_int),
    "gbsz_server_submit_decompress": ([_P, _P, C.c_size_t, _P, C.c_uint64, C.POINTER(C.c_uint64)], C.c_int),
    "gbsz_server_poll": ([_P, C.c_uint64, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_size_t)], C.c_int),
    "gbsz_server_wait": ([_P, C.c_uint64, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_size_t)], C.c_int),
    "gbsz_server_stats": ([_P, _P], C.c_int),
    "gbsz_server_memory": ([_P, _P], C.c_int),
    "gbsz_memory_usage": ([_P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)], C.c_int),
    "gbsz_release_scratch": ([_P], C.c_int),
    "gbsz_tuned_knobs": ([_P, _P, _P], C.c_int),
    "gbsz_scratch_bytes": ([_P, C.c_int, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)], C.c_int),
}
OPT_CODEWORD_BITS = 1
OPT_BATCH_MODE = 3
OPT_DECODER = 4
OPT_LORENZO_SLAB = 5
OPT_TEST_HOLD_CHUNK = 6


class GbszError(RuntimeError):
    def __init__(self, status, what):
        msg = status_str(status) if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} ({status})")
        self.status = status


class Params(C.Structure):
    _fields_ = [("ndim", C.c_uint32), ("dims", C.c_uint64 * 4), ("eb", C.c_double),
                ("eb_mode", C.c_uint32), ("radius", C.c_uint32), ("chunk", C.c_uint32),
                ("lorenzo_block", C.c_uint32), ("lorenzo_order", C.c_uint32)]


_lib = None


def load():
    """Load libgbsz.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is not built; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def status_str(s):
    return load().gbsz_status_str(int(s)).decode()


def make_params(dims, eb, eb_mode=EB_REL, radius=512, chunk=0, lblock=0, order=1):
    """dims: extents with the fastest-varying first (x, y, z, w; a 4D field
    is predicted as 3D with z and w folded).  lblock = 1: Lorenzo inside the
    paper's blocks (see gbsz_params.lorenzo_block); order: Lorenzo order n."""
    dims = [int(d) for d in dims]
    p = Params()
    p.ndim = len(dims)
    for i in range(4):
        p.dims[i] = dims[i] if i < len(dims) else 1
    p.eb, p.eb_mode, p.radius, p.chunk = float(eb), int(eb_mode), int(radius), int(chunk)
    p.lorenzo_block = int(lblock)
    p.lorenzo_order = int(order)
    return p


def field_dims(t):
    """Extents of a C-ordered tensor, fastest first."""
    return list(t.shape)[::-1]


def compress_bound(dims, eb=1e-4, eb_mode=EB_REL, radius=512, chunk=0, lblock=0, order=1):
    return load().gbsz_compress_bound(C.byref(make_params(dims, eb, eb_mode, radius, chunk, lblock, order)))


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Context:
    """A device context; owns resident scratch (see gbsz_create)."""

    def __init__(self, device=0):
        L = load()
        self.device = int(device)
        h = C.c_void_p()
        st = L.gbsz_create(C.byref(h), self.device)
        if st != OK:
            raise GbszError(st, "gbsz_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().gbsz_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- device-buffer API -------------------------------------------------
    def compress(self, field, eb, eb_mode=EB_REL, radius=512, chunk=0, out=None, stream=None, lblock=0,
                 order=1):
        """field: contiguous float32 CUDA tensor (C order, last axis fastest).
        Returns (archive uint8 tensor on the device, nbytes)."""
        assert field.is_cuda and field.dtype == torch.float32 and field.is_contiguous()
        p = make_params(field_dims(field), eb, eb_mode, radius, chunk, lblock, order)
        cap = load().gbsz_compress_bound(C.byref(p))
        if cap == 0:
            raise GbszError(ERR_INVALID_ARG, "compress_bound")
        if out is None:
            out = torch.empty(cap, dtype=torch.uint8, device=field.device)
        nbytes = C.c_size_t()
        st = load().gbsz_compress(self.h, C.c_void_p(field.data_ptr()), C.byref(p),
                                  C.c_void_p(out.data_ptr()), out.numel(), C.byref(nbytes), _stream(stream))
        if st != OK:
            raise GbszError(st, "gbsz_compress")
        return out, nbytes.value

    def autotune(self, field, eb, eb_mode=EB_REL, radius=512, lblock=0, stream=None, order=1):
        """Measured chunk choice for this field's (rank, dims, radius) (see
        gbsz_autotune).  Returns (Params with the chosen chunk, ms)."""
        p = make_params(field_dims(field), eb, eb_mode, radius, 0, lblock, order)
        out = Params()
        ms = C.c_float()
        st = load().gbsz_autotune(self.h, C.c_void_p(field.data_ptr()), C.byref(p), C.byref(out), C.byref(ms),
                                  _stream(stream))
        if st != OK:
            raise GbszError(st, "gbsz_autotune")
        return out, ms.value

    def tuned_knobs(self, params):
        """(chunk, decoder, slab) that autotune chose for params' key (see
        gbsz_tuned_knobs)."""
        k = (C.c_uint32 * 3)()
        st = load().gbsz_tuned_knobs(self.h, C.byref(params), k)
        if st != OK:
            raise GbszError(st, "gbsz_tuned_knobs")
        return tuple(k)

    def compress_params(self, field, params, out=None, stream=None):
        """Compress with an explicit Params (e.g. from autotune)."""
        cap = load().gbsz_compress_bound(C.byref(params))
        if out is None:
            out = torch.empty(cap, dtype=torch.uint8, device=field.device)
        st, nb = self.compress_status(field, params, out, stream)
        if st != OK:
            raise GbszError(st, "gbsz_compress")
        return out, nb

    def compress_status(self, field, params, out, stream=None):
        """Raw status call: returns (status, nbytes) without raising."""
        nbytes = C.c_size_t()
        st = load().gbsz_compress(self.h, C.c_void_p(field.data_ptr()), C.byref(params),
                                  C.c_void_p(out.data_ptr()), out.numel(), C.byref(nbytes), _stream(stream))
        return st, nbytes.value

    def decompress(self, archive, nbytes=None, out=None, stream=None):
        """archive: uint8 CUDA tensor.  Returns the float32 field tensor."""
        nbytes = archive.numel() if nbytes is None else int(nbytes)
        if out is None:
            hdr = archive[:128].cpu().numpy()
            p, n = archive_info(hdr, nbytes)
            shape = [int(p.dims[i]) for i in range(p.ndim)][::-1]
            out = torch.empty(shape, dtype=torch.float32, device=archive.device)
        st = load().gbsz_decompress(self.h, C.c_void_p(archive.data_ptr()), nbytes,
                                    C.c_void_p(out.data_ptr()), out.numel(), _stream(stream))
        if st != OK:
            raise GbszError(st, "gbsz_decompress")
        return out

    def decompress_status(self, archive, nbytes, out, stream=None):
        return load().gbsz_decompress(self.h, C.c_void_p(archive.data_ptr()), int(nbytes),
                                      C.c_void_p(out.data_ptr()), out.numel(), _stream(stream))

    # -- batches -------------------------------------------------------------
    def compress_batch(self, fields, eb, eb_mode=EB_REL, radius=512, chunk=0, outs=None, stream=None,
                       params=None):
        """fields: list of contiguous float32 CUDA tensors.  eb/radius/chunk
        may be scalars or per-field lists.  Returns (list of archive tensors,
        list of nbytes, list of statuses); raises if any field failed."""
        k = len(fields)
        per = lambda v: list(v) if isinstance(v, (list, tuple)) else [v] * k
        ebs, rads, chunks, modes = per(eb), per(radius), per(chunk), per(eb_mode)
        if params is None:
            params = [make_params(field_dims(f), e, m, r, c) for f, e, m, r, c in zip(fields, ebs, modes, rads, chunks)]
        P = (Params * k)(*params)
        if outs is None:
            outs = [torch.empty(load().gbsz_compress_bound(C.byref(p)), dtype=torch.uint8, device=f.device)
                    for p, f in zip(params, fields)]
        fp = (C.c_void_p * k)(*[f.data_ptr() for f in fields])
        ap = (C.c_void_p * k)(*[o.data_ptr() for o in outs])
        caps = (C.c_size_t * k)(*[o.numel() for o in outs])
        nb = (C.c_size_t * k)()
        sts = (C.c_int * k)()
        st = load().gbsz_compress_batch(self.h, k, fp, P, ap, caps, nb, sts, _stream(stream))
        if st != OK:
            raise GbszError(st, "gbsz_compress_batch")
        return outs, list(nb), list(sts)

    def decompress_batch(self, archives, nbytes, outs, stream=None):
        """archives: list of uint8 CUDA tensors; outs: float32 CUDA tensors."""
        k = len(archives)
        ap = (C.c_void_p * k)(*[a.data_ptr() for a in archives])
        bs = (C.c_size_t * k)(*[int(b) for b in nbytes])
        op = (C.c_void_p * k)(*[o.data_ptr() for o in outs])
        caps = (C.c_uint64 * k)(*[o.numel() for o in outs])
        sts = (C.c_int * k)()
        st = load().gbsz_decompress_batch(self.h, k, ap, bs, op, caps, sts, _stream(stream))
        if st != OK:
            raise GbszError(st, "gbsz_decompress_batch")
        return outs, list(sts)

    def memory_usage(self):
        """(device bytes the context holds, its scratch slots)."""
        b, k = C.c_uint64(), C.c_uint32()
        st = load().gbsz_memory_usage(self.h, C.byref(b), C.byref(k))
        if st != OK:
            raise GbszError(st, "gbsz_memory_usage")
        return b.value, k.value

    def release_scratch(self):
        st = load().gbsz_release_scratch(self.h)
        if st != OK:
            raise GbszError(st, "gbsz_release_scratch")

    def set_option(self, option, value):
        st = load().gbsz_set_option(self.h, int(option), int(value))
        if st != OK:
            raise GbszError(st, "gbsz_set_option")

    # -- host-buffer API ---------------------------------------------------
    def compress_host(self, field_np, eb, eb_mode=EB_REL, radius=512, chunk=0, out=None, stream=None,
                      lblock=0):
        """field_np: contiguous float32 numpy array (or pinned CPU tensor)."""
        import numpy as np
        ptr, shape = _host_ptr(field_np)
        p = make_params(shape[::-1], eb, eb_mode, radius, chunk, lblock)
        cap = load().gbsz_compress_bound(C.byref(p))
        if out is None:
            out = np.empty(cap, dtype=np.uint8)
        optr, _ = _host_ptr(out)
        nbytes = C.c_size_t()
        st = load().gbsz_compress_host(self.h, ptr, C.byref(p), optr, _nbytes(out), C.byref(nbytes),
                                       _stream(stream))
        if st != OK:
            raise GbszError(st, "gbsz_compress_host")
        return out, nbytes.value

    def decompress_host_async(self, archive, nbytes, out, stream=None):
        """Enqueue a host-buffer decompress and return at once (see
        gbsz_decompress_host_async); async_wait() reports its status."""
        aptr, _ = _host_ptr(archive)
        optr, _ = _host_ptr(out)
        st = load().gbsz_decompress_host_async(self.h, aptr, int(nbytes), optr, _numel(out), _stream(stream))
        if st != OK:
            raise GbszError(st, "gbsz_decompress_host_async")

    def async_wait(self):
        st = load().gbsz_async_wait(self.h)
        if st != OK:
            raise GbszError(st, "gbsz_async_wait")

    def decompress_host(self, archive, nbytes, out, stream=None):
        aptr, _ = _host_ptr(archive)
        optr, _ = _host_ptr(out)
        st = load().gbsz_decompress_host(self.h, aptr, int(nbytes), optr, _numel(out), _stream(stream))
        if st != OK:
            raise GbszError(st, "gbsz_decompress_host")
        return out

    # -- introspection -----------------------------------------------------
    def debug_copy(self, which, count, dtype):
        import numpy as np
        a = np.zeros(count, dtype=dtype)
        st = load().gbsz_debug_copy(self.h, int(which), C.c_void_p(a.ctypes.data), a.nbytes)
        if st != OK:
            raise GbszError(st, "gbsz_debug_copy")
        return a

    def profile_enable(self, on=True):
        load().gbsz_profile_enable(self.h, 1 if on else 0)

    def profile_read(self):
        """Returns (stage_ms[8], stage_calls[8], kernel_launches)."""
        ms = (C.c_double * NSTAGE)()
        calls = (C.c_uint64 * NSTAGE)()
        kl = C.c_uint64()
        st = load().gbsz_profile_read(self.h, C.cast(ms, C.c_void_p), C.cast(calls, C.c_void_p), C.byref(kl))
        if st != OK:
            raise GbszError(st, "gbsz_profile_read")
        return list(ms), list(calls), kl.value


def _host_ptr(a):
    if isinstance(a, torch.Tensor):
        assert not a.is_cuda and a.is_contiguous()
        return C.c_void_p(a.data_ptr()), list(a.shape)
    assert a.flags["C_CONTIGUOUS"]
    return C.c_void_p(a.ctypes.data), list(a.shape)


def _nbytes(a):
    return a.numel() * a.element_size() if isinstance(a, torch.Tensor) else a.nbytes


def _numel(a):
    return a.numel() if isinstance(a, torch.Tensor) else a.size


def archive_info(header_bytes, nbytes=None):
    """Parse a host copy of the archive header (numpy uint8).  Returns (Params, n)."""
    import numpy as np
    h = np.ascontiguousarray(header_bytes, dtype=np.uint8)
    nb = int(nbytes) if nbytes is not None else h.size
    p = Params()
    n = C.c_uint64()
    st = load().gbsz_archive_info(C.c_void_p(h.ctypes.data), nb, C.byref(p), C.byref(n))
    if st != OK:
        raise GbszError(st, "gbsz_archive_info")
    return p, n.value


def scratch_bytes(dims, eb=1e-4, eb_mode=EB_REL, radius=512, chunk=0, lblock=0, order=1, for_decompress=False):
    """(scratch one such field adds to a context slot, fixed bytes of one slot)."""
    f, sl = C.c_uint64(), C.c_uint64()
    st = load().gbsz_scratch_bytes(C.byref(make_params(dims, eb, eb_mode, radius, chunk, lblock, order)),
                                   1 if for_decompress else 0, C.byref(f), C.byref(sl))
    if st != OK:
        raise GbszError(st, "gbsz_scratch_bytes")
    return f.value, sl.value


def auto_chunk(dims, radius=512):
    return load().gbsz_auto_chunk(C.byref(make_params(dims, 1e-4, EB_REL, radius, 0)))


def codebook_noalloc(hist, stream=None, out=None):
    """Code lengths and canonical codewords from a device histogram, through
    the entry point that allocates no device memory (see gbsz.h).  The output
    tensors are allocated here by torch unless `out` = (lengths, codewords,
    ...) from an earlier call is given; the library allocates nothing."""
    assert hist.is_cuda and hist.dtype == torch.int32 and hist.is_contiguous()
    nb = hist.numel()
    if out is not None:
        ln, code = out[0], out[1]
        assert ln.numel() == nb and code.numel() == nb and ln.dtype == torch.uint8 and code.dtype == torch.int64
    else:
        ln = torch.empty(nb, dtype=torch.uint8, device=hist.device)
        code = torch.empty(nb, dtype=torch.int64, device=hist.device)
    mx = C.c_uint32()
    st = load().gbsz_codebook_noalloc(C.c_void_p(hist.data_ptr()), nb, C.c_void_p(ln.data_ptr()),
                                      C.c_void_p(code.data_ptr()), C.byref(mx), _stream(stream))
    if st != OK:
        raise GbszError(st, "gbsz_codebook_noalloc")
    return ln, code, mx.value
