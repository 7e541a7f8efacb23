"""The OpenMP build of the oracle (the multi-core CPU baseline) restates the
serial loops over chunks, over the outlier list and over the reconstruction
cascade in independent pieces.  It must give the single-threaded build's
bytes, reconstructions and statuses exactly, on every mode: 1D / 2D / 3D / 4D
fields, Lorenzo orders 1-3, the per-block mode, ragged chunk tails, fields
with non-finite values, and corrupt archives."""
import numpy as np
import pytest

from oracle import ref
from paper_2007_09625_gb300 import workloads

CASES = [
    # (kind, shape, rel, radius, chunk, lblock, order)
    ("walk", (300007,), 1e-4, 512, 256, 0, 1),
    ("walk", (300007,), 1e-4, 512, 2048, 0, 1),  # chunk anchors
    ("walk", (300007,), 1e-4, 512, 4096, 1, 1),
    ("walk", (100003,), 1e-3, 64, 128, 0, 2),
    ("walk", (100003,), 1e-3, 512, 1024, 0, 3),
    ("grf", (181, 1037), 1e-4, 512, 512, 0, 1),
    ("grf", (181, 1037), 1e-3, 512, 64, 1, 1),
    ("grf", (97, 301), 1e-3, 512, 256, 0, 2),
    ("lognormal", (37, 41, 67), 1e-4, 512, 2048, 0, 1),
    ("lognormal", (37, 41, 67), 1e-5, 32768, 4096, 0, 1),
    ("lognormal", (19, 23, 29), 1e-3, 512, 256, 1, 1),
    ("lognormal", (19, 23, 29), 1e-3, 512, 256, 0, 3),
    ("sinus", (6, 7, 9, 11), 1e-4, 512, 64, 0, 1),
]


@pytest.mark.parametrize("kind,shape,rel,R,chunk,lblock,order", CASES)
def test_omp_build_equals_single_thread(kind, shape, rel, R, chunk, lblock, order):
    if kind == "sinus":
        x = workloads.field_for("sinus", shape[1:], seed=41).reshape(1, *shape[1:])
        x = np.concatenate([x * (1 + 0.1 * k) for k in range(shape[0])]).astype(np.float32)
    else:
        x = workloads.field_for(kind, shape, seed=40 + len(shape))
    a1 = ref.compress(x, rel, ref.EB_REL, R, chunk, lblock=lblock, order=order)
    a2 = ref.compress(x, rel, ref.EB_REL, R, chunk, omp=True, lblock=lblock, order=order)
    assert np.array_equal(a1, a2)
    y1 = ref.decompress(a1)
    y2 = ref.decompress(a1, omp=True)
    assert np.array_equal(y1.view(np.uint32), y2.view(np.uint32))


def test_omp_build_nonfinite_and_constant():
    rng = np.random.default_rng(44)
    x = rng.normal(0, 1, 70001).astype(np.float32)
    x[::997] = np.nan
    x[5] = np.inf
    x[77] = np.float32(3e38)
    for f in (x, np.full(5000, 2.5, np.float32), np.zeros(1, np.float32)):
        a1 = ref.compress(f, 1e-3, ref.EB_REL, 512, 64)
        a2 = ref.compress(f, 1e-3, ref.EB_REL, 512, 64, omp=True)
        assert np.array_equal(a1, a2)
        assert np.array_equal(ref.decompress(a1).view(np.uint32), ref.decompress(a1, omp=True).view(np.uint32))


def _status(lib, a, cap):
    import ctypes as C
    y = np.zeros(cap, np.float32)
    return lib.gbsz_ref_decompress(a.ctypes.data_as(C.c_void_p), a.size, y.ctypes.data_as(C.c_void_p), cap)


@pytest.mark.parametrize("chunk", [256, 1024])
def test_omp_build_corrupt_archives_same_status(chunk):
    rng = np.random.default_rng(45)
    x = np.cumsum(rng.normal(0, 1, 20000)).astype(np.float32)
    a = ref.compress(x, 1e-4, chunk=chunk)
    s = ref.sections(a)
    st, om = ref.lib(), ref.lib(omp=True)
    cases = []
    for t in range(300):  # random byte flips past the header
        b = a.copy()
        b[int(rng.integers(128, a.size))] ^= np.uint8(1 << int(rng.integers(0, 8)))
        cases.append(b)
    if s["m"] >= 2:  # outlier list out of order, and pointing at a nonzero code
        o = s["off_out"]
        b = a.copy()
        b[o:o + 4], b[o + 8:o + 12] = a[o + 8:o + 12].copy(), a[o:o + 4].copy()
        cases.append(b)
        b = a.copy()
        idx = int(a[o:o + 4].view(np.uint32)[0])
        b[o:o + 4] = np.array([idx + 1 if idx + 1 < x.size else idx - 1], np.uint32).view(np.uint8)
        cases.append(b)
    for c in range(s["nanchor"]):  # every anchor off by one
        b = a.copy()
        b[s["off_anc"] + 4 * c:s["off_anc"] + 4 * c + 4] = (s["anchors"][c:c + 1] + np.uint32(1)).view(np.uint8)
        cases.append(b)
    for b in cases:
        assert _status(st, b, x.size) == _status(om, b, x.size)


def test_omp_reconstruct_rejects_what_serial_rejects():
    """Direct calls with an outlier list that does not match the code-0 points."""
    codes = np.array([512, 0, 513, 0, 511, 512], np.uint16)
    good = (np.array([1, 3], np.uint32), np.array([7, -9], np.int32))
    bads = [(np.array([1], np.uint32), np.array([7], np.int32)),             # too few
            (np.array([1, 2], np.uint32), np.array([7, -9], np.int32)),      # names a nonzero code
            (np.array([3, 1], np.uint32), np.array([7, -9], np.int32)),      # out of order
            (np.array([1, 3, 5], np.uint32), np.array([7, -9, 1], np.int32))]  # too many
    empty = (np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    for idx, dl in [good] + bads:
        outs = []
        for omp in (False, True):
            import ctypes as C
            L = ref.lib(omp)
            y = np.zeros(codes.size, np.float32)
            dims = np.array([codes.size, 1, 1], np.uint64)
            p = lambda a: a.ctypes.data_as(C.c_void_p)
            r = L.gbsz_ref_reconstruct(p(codes), 1, p(dims), 512, p(idx), p(dl), idx.size, p(empty[0]),
                                       p(empty[1]), 0, C.c_float(0.5), p(y))
            outs.append((r, y.copy()))
        assert outs[0][0] == outs[1][0]
        if outs[0][0] == 0:
            assert np.array_equal(outs[0][1].view(np.uint32), outs[1][1].view(np.uint32))
