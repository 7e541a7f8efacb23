"""ctypes bindings of the C oracle (test infrastructure only).

Every function takes and returns numpy arrays in host memory and raises
``OracleError`` on a non-zero status.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_CORRUPT, ERR_OOM = 0, 1, 2, 3, 4
EB_ABS, EB_REL = 0, 1


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: oracle status {status}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("ndim", C.c_uint32), ("dims", C.c_uint64 * 4), ("eb", C.c_double),
                ("eb_mode", C.c_uint32), ("radius", C.c_uint32), ("chunk", C.c_uint32),
                ("lorenzo_block", C.c_uint32), ("lorenzo_order", C.c_uint32)]


def make_params(dims, eb, eb_mode=EB_REL, radius=512, chunk=4096, lblock=0, order=1):
    dims = tuple(int(d) for d in dims)
    p = Params()
    p.ndim = len(dims)
    for i in range(4):
        p.dims[i] = dims[i] if i < len(dims) else 1
    p.eb, p.eb_mode, p.radius, p.chunk = float(eb), int(eb_mode), int(radius), int(chunk)
    p.lorenzo_block = int(lblock)
    p.lorenzo_order = int(order)
    return p


_lib = {}


def lib(omp=False):
    key = "omp" if omp else "st"
    if key not in _lib:
        _build.build()
        L = C.CDLL(_build.LIB_OMP if omp else _build.LIB)
        P = C.c_void_p
        u32, u64 = C.c_uint32, C.c_uint64
        sig = {
            "gbsz_ref_threads": [],
            "gbsz_ref_error_bound": [P, u64, u32, C.c_double, P],
            "gbsz_ref_prequant_one": [C.c_float, P, P],
            "gbsz_ref_lorenzo_delta": [P, u32, P, u32, P],
            "gbsz_ref_lorenzo_delta_blocked": [P, u32, P, u32, u32, P],
            "gbsz_ref_dualquant": [P, u32, P, P, u32, P, P, P, P, P, P, P, P],
            "gbsz_ref_dualquant_ex": [P, u32, P, P, u32, u32, u32, P, P, P, P, P, P, P, P],
            "gbsz_ref_histogram": [P, u64, u32, P],
            "gbsz_ref_huffman_lengths": [P, u32, P, P],
            "gbsz_ref_canonical_codes": [P, u32, P],
            "gbsz_ref_deflate": [P, u64, u32, P, P, P, P, u64, P],
            "gbsz_ref_inflate": [P, u64, P, u64, u32, P, u32, P],
            "gbsz_ref_reconstruct": [P, u32, P, u32, P, P, u64, P, P, u64, C.c_float, P],
            "gbsz_ref_reconstruct_ex": [P, u32, P, u32, u32, u32, P, P, u64, P, P, u64, C.c_float, P],
            "gbsz_ref_compress": [P, P, P, C.c_size_t, P],
            "gbsz_ref_decompress": [P, C.c_size_t, P, u64],
            "gbsz_ref_archive_info": [P, C.c_size_t, P, P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.gbsz_ref_compress_bound.argtypes = [P]
        L.gbsz_ref_compress_bound.restype = C.c_size_t
        L.gbsz_ref_lorenzo_block_extent.argtypes = [u32]
        L.gbsz_ref_lorenzo_block_extent.restype = u32
        _lib[key] = L
    return _lib[key]


def threads(omp=False):
    """Threads the given build's parallel loops use."""
    return lib(omp).gbsz_ref_threads()


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _dims3(dims):
    d = np.ones(3, dtype=np.uint64)
    d[:len(dims)] = dims
    return d


def _check(st, what):
    if st != OK:
        raise OracleError(st, what)


def error_bound(x, eb, eb_mode=EB_REL):
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    out = np.zeros(3, dtype=np.float32)
    _check(lib().gbsz_ref_error_bound(_p(x), x.size, eb_mode, eb, _p(out)), "error_bound")
    return out


def prequant_one(x, sc):
    sc = np.ascontiguousarray(sc, dtype=np.float32)
    q = C.c_int32()
    exc = lib().gbsz_ref_prequant_one(C.c_float(float(x)), _p(sc), C.byref(q))
    return int(q.value), bool(exc)


def lorenzo_delta(q, order=1, lblock=0):
    q = np.ascontiguousarray(q, dtype=np.int32)
    dims = q.shape[::-1]  # numpy C order: last axis varies fastest
    out = np.zeros_like(q)
    if lblock:
        st = lib().gbsz_ref_lorenzo_delta_blocked(_p(q), len(dims), _p(_dims3(dims)), order, lblock, _p(out))
    else:
        st = lib().gbsz_ref_lorenzo_delta(_p(q), len(dims), _p(_dims3(dims)), order, _p(out))
    _check(st, "lorenzo_delta")
    return out


def lorenzo_block_extent(ndim):
    return int(lib().gbsz_ref_lorenzo_block_extent(ndim))


def dualquant(x, sc, radius, lblock=0, order=1):
    """Returns dict(codes, out_idx, out_delta, exc_idx, exc_raw, q)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    dims = x.shape[::-1]
    n = x.size
    sc = np.ascontiguousarray(sc, dtype=np.float32)
    codes = np.zeros(n, np.uint16)
    oi, od = np.zeros(n, np.uint32), np.zeros(n, np.int32)
    ei, er = np.zeros(n, np.uint32), np.zeros(n, np.uint32)
    q = np.zeros(n, np.int32)
    m, e = C.c_uint64(), C.c_uint64()
    _check(lib().gbsz_ref_dualquant_ex(_p(x), len(dims), _p(_dims3(dims)), _p(sc), radius, lblock, order,
                                       _p(codes), _p(oi), _p(od), C.byref(m), _p(ei), _p(er),
                                       C.byref(e), _p(q)), "dualquant")
    m, e = m.value, e.value
    return dict(codes=codes, out_idx=oi[:m].copy(), out_delta=od[:m].copy(),
                exc_idx=ei[:e].copy(), exc_raw=er[:e].copy(), q=q)


def histogram(codes, nbins):
    codes = np.ascontiguousarray(codes, dtype=np.uint16)
    h = np.zeros(nbins, np.uint32)
    _check(lib().gbsz_ref_histogram(_p(codes), codes.size, nbins, _p(h)), "histogram")
    return h


def huffman_lengths(hist):
    hist = np.ascontiguousarray(hist, dtype=np.uint32)
    ln = np.zeros(hist.size, np.uint8)
    mx = C.c_uint32()
    _check(lib().gbsz_ref_huffman_lengths(_p(hist), hist.size, _p(ln), C.byref(mx)),
           "huffman_lengths")
    return ln, mx.value


def canonical_codes(lengths):
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    code = np.zeros(lengths.size, np.uint64)
    _check(lib().gbsz_ref_canonical_codes(_p(lengths), lengths.size, _p(code)), "canonical")
    return code


def deflate(codes, chunk, lengths, code):
    codes = np.ascontiguousarray(codes, dtype=np.uint16)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    code = np.ascontiguousarray(code, dtype=np.uint64)
    n = codes.size
    nc = (n + chunk - 1) // chunk
    cap = nc + (45 * n + 31) // 32
    bits = np.zeros(nc, np.uint32)
    stream = np.zeros(max(cap, 1), np.uint32)
    w = C.c_uint64()
    _check(lib().gbsz_ref_deflate(_p(codes), n, chunk, _p(lengths), _p(code), _p(bits),
                                  _p(stream), cap, C.byref(w)), "deflate")
    return bits, stream[:w.value].copy()


def inflate(stream, bits, n, chunk, lengths):
    stream = np.ascontiguousarray(stream, dtype=np.uint32)
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    lengths = np.ascontiguousarray(lengths, dtype=np.uint8)
    codes = np.zeros(n, np.uint16)
    _check(lib().gbsz_ref_inflate(_p(stream), stream.size, _p(bits), n, chunk, _p(lengths),
                                  lengths.size, _p(codes)), "inflate")
    return codes


def reconstruct(codes, dims, radius, out_idx, out_delta, exc_idx, exc_raw, ebx2, lblock=0, order=1):
    """dims in numpy order (slowest first); returns float32 array of that shape."""
    codes = np.ascontiguousarray(codes, dtype=np.uint16).ravel()
    fd = tuple(dims)[::-1]
    oi = np.ascontiguousarray(out_idx, dtype=np.uint32)
    od = np.ascontiguousarray(out_delta, dtype=np.int32)
    ei = np.ascontiguousarray(exc_idx, dtype=np.uint32)
    er = np.ascontiguousarray(exc_raw, dtype=np.uint32)
    x = np.zeros(codes.size, np.float32)
    _check(lib().gbsz_ref_reconstruct_ex(_p(codes), len(fd), _p(_dims3(fd)), radius, lblock, order, _p(oi),
                                         _p(od), oi.size, _p(ei), _p(er), ei.size, C.c_float(ebx2), _p(x)),
           "reconstruct")
    return x.reshape(dims)


def compress_bound(shape, eb, eb_mode=EB_REL, radius=512, chunk=4096, lblock=0, order=1):
    p = make_params(tuple(shape)[::-1], eb, eb_mode, radius, chunk, lblock, order)
    return lib().gbsz_ref_compress_bound(C.byref(p))


def compress(x, eb, eb_mode=EB_REL, radius=512, chunk=4096, omp=False, lblock=0, order=1):
    """x: numpy float32 array, C order (last axis fastest; up to 4 axes, a 4D
    field being predicted as 3D with its two slowest axes folded).  Returns
    bytes array.  lblock = 1: Lorenzo inside the paper's blocks (zero padding
    layer); order: Lorenzo order n (1..3)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    p = make_params(x.shape[::-1], eb, eb_mode, radius, chunk, lblock, order)
    L = lib(omp)
    cap = L.gbsz_ref_compress_bound(C.byref(p))
    if cap == 0:
        raise OracleError(ERR_INVALID_ARG, "compress_bound")
    buf = np.zeros(cap, np.uint8)
    nbytes = C.c_size_t()
    _check(L.gbsz_ref_compress(_p(x), C.byref(p), _p(buf), cap, C.byref(nbytes)), "compress")
    return buf[:nbytes.value].copy()


def archive_info(archive):
    a = np.ascontiguousarray(archive, dtype=np.uint8)
    p = Params()
    n = C.c_uint64()
    _check(lib().gbsz_ref_archive_info(_p(a), a.size, C.byref(p), C.byref(n)), "archive_info")
    return p, n.value


def decompress(archive, omp=False):
    a = np.ascontiguousarray(archive, dtype=np.uint8)
    p, n = archive_info(a)
    x = np.zeros(n, np.float32)
    _check(lib(omp).gbsz_ref_decompress(_p(a), a.size, _p(x), n), "decompress")
    dims = tuple(int(p.dims[i]) for i in range(p.ndim))[::-1]
    return x.reshape(dims)


def decompress_status(archive, capacity=None):
    """Raw status of a decompress (for corrupt-archive tests)."""
    a = np.ascontiguousarray(archive, dtype=np.uint8)
    cap = capacity if capacity is not None else 1 << 22
    x = np.zeros(cap, np.float32)
    return lib().gbsz_ref_decompress(_p(a), a.size, _p(x), cap)


# archive section helpers (the format, restated for the tests' field access)
HEADER = 128
ANCHOR_CHUNK = 1024


def sections(archive):
    """Parse header fields and section offsets from raw bytes."""
    a = np.ascontiguousarray(archive, dtype=np.uint8)
    b = a.tobytes()
    u32 = lambda o: int.from_bytes(b[o:o + 4], "little")
    u64 = lambda o: int.from_bytes(b[o:o + 8], "little")
    R, nc, m, e, w = u32(68), u32(76), u64(80), u64(88), u64(96)
    al = lambda v: (v + 15) & ~15
    # chunk anchors: 1D, one order-1 predictor, chunks of at least 1024 symbols
    na = nc if (u32(8) == 1 and u32(120) <= 1 and u32(108) == 0 and u32(72) >= ANCHOR_CHUNK) else 0
    off_len = HEADER
    off_bits = al(off_len + 2 * R)
    off_anc = al(off_bits + 4 * nc)
    off_out = al(off_anc + 4 * na)
    off_exc = off_out + 8 * m
    off_str = al(off_exc + 8 * e)
    d = dict(radius=R, nchunk=nc, m=m, e=e, words=w, maxlen=u32(104), chunk=u32(72), lblock=u32(108),
             total=u64(112), n=u64(40), order=u32(120), ndim=u32(8),
             sc=np.frombuffer(b[56:68], dtype=np.float32).copy(),
             off_len=off_len, off_bits=off_bits, off_anc=off_anc, off_out=off_out, off_exc=off_exc,
             off_str=off_str, nanchor=na)
    d["len"] = a[off_len:off_len + 2 * R].copy()
    d["bits"] = np.frombuffer(b[off_bits:off_bits + 4 * nc], np.uint32).copy()
    d["anchors"] = np.frombuffer(b[off_anc:off_anc + 4 * na], np.uint32).copy()
    o = np.frombuffer(b[off_out:off_out + 8 * m], np.uint32).reshape(-1, 2)
    d["out_idx"], d["out_delta"] = o[:, 0].copy(), o[:, 1].view(np.int32).copy()
    ex = np.frombuffer(b[off_exc:off_exc + 8 * e], np.uint32).reshape(-1, 2)
    d["exc_idx"], d["exc_raw"] = ex[:, 0].copy(), ex[:, 1].copy()
    d["stream"] = np.frombuffer(b[off_str:off_str + 4 * w], np.uint32).copy()
    return d
