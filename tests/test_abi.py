"""The C-ABI library loads without a GPU, exports every symbol include/gbsz.h
declares, and its host-only entry points behave (no device work here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2007_09625_gb300 import build as lib_build
from paper_2007_09625_gb300 import gbsz

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    lib_build.build()
    return gbsz.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gbsz.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gbsz_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
        assert name in gbsz.SIGNATURES, f"binding lacks {name}"


def test_status_strings(lib):
    for s in range(8):
        assert gbsz.status_str(s)
    assert gbsz.status_str(3) == "corrupt archive"


def test_compress_bound_and_invalid_params(lib):
    p = gbsz.make_params([1 << 20], 1e-4, gbsz.EB_REL, 512, 4096)
    b = lib.gbsz_compress_bound(C.byref(p))
    n = 1 << 20
    # header and padding, lengths, chunk bits and anchors, 16 B a point, the longest stream
    assert b == 208 + 1024 + 12 * 256 + 16 * n + 4 * (256 + (45 * n + 31) // 32)
    for bad in (dict(dims=[0]), dict(dims=[1 << 32]), dict(dims=[1 << 16, 1 << 16]),
                dict(eb=0.0), dict(eb=float("nan")), dict(radius=1), dict(radius=32769),
                dict(chunk=32), dict(chunk=100), dict(chunk=131072)):
        kw = dict(dims=[1000], eb=1e-4, radius=512, chunk=4096)
        kw.update(bad)
        q = gbsz.make_params(kw["dims"], kw["eb"], gbsz.EB_REL, kw["radius"], kw["chunk"])
        assert lib.gbsz_compress_bound(C.byref(q)) == 0, bad


def test_auto_chunk_rule(lib):
    # smallest power of two (64..4096) with n <= chunk * 1024 * 152
    assert gbsz.auto_chunk([1 << 28]) == 2048
    assert gbsz.auto_chunk([2048 * 1024 * 152]) == 2048
    assert gbsz.auto_chunk([2048 * 1024 * 152 + 1]) == 4096
    assert gbsz.auto_chunk([1 << 30]) == 4096
    assert gbsz.auto_chunk([64, 64, 64]) == 64
    assert gbsz.auto_chunk([512, 512, 512]) == 1024
    assert gbsz.auto_chunk([3600, 1800]) == 64


def test_bench_chunk_rule_matches_library(lib):
    """The benchmark restates the rule so that its reference arm runs the same
    configuration without the library; both must agree for every n."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    rng = np.random.default_rng(5)
    ns = [1, 63, 64, 155648, 155649, 64 * 155648, 64 * 155648 + 1, 1 << 26, 1 << 28, (1 << 32) - 1]
    ns += [int(v) for v in rng.integers(1, 1 << 32, 200)]
    for n in ns:
        assert bench.workload_chunk(n) == gbsz.auto_chunk([n]), n


def test_null_context_and_pointers_rejected(lib):
    nb = C.c_size_t()
    p = gbsz.make_params([10], 1e-3)
    assert lib.gbsz_compress(None, None, C.byref(p), None, 0, C.byref(nb), None) == gbsz.ERR_INVALID_ARG
    assert lib.gbsz_decompress(None, None, 0, None, 0, None) == gbsz.ERR_INVALID_ARG
    assert lib.gbsz_create(None, 0) == gbsz.ERR_INVALID_ARG
    assert lib.gbsz_profile_enable(None, 1) == gbsz.ERR_INVALID_ARG


def test_archive_info_parses_oracle_archives(lib, oracle):
    rng = np.random.default_rng(0)
    x = rng.normal(size=(7, 9, 11)).astype(np.float32)
    a = oracle.compress(x, 1e-3, oracle.EB_REL, radius=64, chunk=128)
    p, n = gbsz.archive_info(a, a.size)
    assert n == x.size and p.ndim == 3 and list(p.dims) == [11, 9, 7, 1]
    assert p.radius == 64 and p.chunk == 128 and p.eb_mode == gbsz.EB_REL and p.lorenzo_order == 1
    x4 = rng.normal(size=(2, 3, 5, 7)).astype(np.float32)
    a4 = oracle.compress(x4, 1e-3, oracle.EB_REL, radius=64, chunk=64, order=2)
    p4, n4 = gbsz.archive_info(a4, a4.size)
    assert n4 == x4.size and p4.ndim == 4 and list(p4.dims) == [7, 5, 3, 2] and p4.lorenzo_order == 2
    for order in (0, 4):  # stored orders are 1..3
        bad = a4.copy()
        bad[120:124] = np.frombuffer(np.uint32(order).tobytes(), np.uint8)
        with pytest.raises(gbsz.GbszError):
            gbsz.archive_info(bad, bad.size)
    bad = a.copy()
    bad[0] ^= 1
    with pytest.raises(gbsz.GbszError):
        gbsz.archive_info(bad, bad.size)
    with pytest.raises(gbsz.GbszError):
        gbsz.archive_info(a, a.size - 1)


def test_archive_info_parses_anchored_archives(lib, oracle):
    """Archives of 1D fields in chunks of at least 1024 symbols carry one
    anchor per chunk between the chunk table and the outliers: the library's
    host-side parser lays the sections out as the oracle wrote them (its total
    size check passes only then), its compress bound covers them, and an
    archive of the previous format version is refused by both."""
    rng = np.random.default_rng(1)
    x = np.cumsum(rng.normal(size=50001)).astype(np.float32)
    for chunk in (512, 1024, 4096, 65536):
        a = oracle.compress(x, 1e-4, oracle.EB_REL, radius=512, chunk=chunk)
        p, n = gbsz.archive_info(a, a.size)
        assert n == x.size and p.chunk == chunk and p.ndim == 1
        nc = (x.size + chunk - 1) // chunk
        assert oracle.sections(a)["nanchor"] == (nc if chunk >= 1024 else 0)
        q = gbsz.make_params([x.size], 1e-4, gbsz.EB_REL, 512, chunk)
        assert lib.gbsz_compress_bound(C.byref(q)) >= a.size
        old = a.copy()
        old[4:6] = np.frombuffer(np.uint16(1).tobytes(), np.uint8)  # format version 1
        with pytest.raises(gbsz.GbszError):
            gbsz.archive_info(old, old.size)
        assert oracle.decompress_status(old) == oracle.ERR_CORRUPT


def test_create_without_gpu_is_a_clean_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.gbsz_create(C.byref(h), 0) == gbsz.ERR_UNSUPPORTED
