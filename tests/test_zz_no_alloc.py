"""gbsz_codebook_noalloc -- the codebook entry point for callers that cannot
allocate device memory (frameworks that own all device memory through their
own pool, processes under a fixed device-memory budget) -- must give the
oracle's code lengths and canonical codewords for the same histogram
(integer results, compared for equality), on two calls in a row, and the
same as the compressor's own codebook stage; once warm, its calls must not
change the free device memory.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest
import torch

from oracle import ref
from paper_2007_09625_gb300 import workloads

pytestmark = pytest.mark.gpu


def compressor_codebook(gb, ctx, x, rel, R):
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    arc, nb = ctx.compress(xt, rel, gb.EB_REL, R, 0)
    hist = ctx.debug_copy(gb.DEBUG_HIST, 2 * R, np.uint32)
    code = ctx.debug_copy(gb.DEBUG_CODEWORDS, 2 * R, np.uint64)
    s = ref.sections(arc[:nb].cpu().numpy())
    return hist, s["len"], code, s["maxlen"]


def test_codebook_noalloc_matches_oracle(gb):
    ctx = gb.Context(0)
    cases = [
        (workloads.field_for("walk", (200003,), seed=21), 1e-4, 512),
        (workloads.field_for("lognormal", (30, 40, 50), seed=22), 1e-5, 32768),
    ]
    for x, rel, R in cases:
        hist, comp_len, comp_code, comp_max = compressor_codebook(gb, ctx, x, rel, R)
        want_len, want_max = ref.huffman_lengths(hist)
        want_code = ref.canonical_codes(want_len)
        h = torch.from_numpy(hist.view(np.int32)).cuda()
        for _ in range(2):  # consecutive calls share the library's scratch
            ln, code, mx = gb.codebook_noalloc(h)
            torch.cuda.synchronize()
            got_len = ln.cpu().numpy()
            got_code = code.cpu().numpy().view(np.uint64)
            assert np.array_equal(got_len, want_len)
            assert np.array_equal(got_code, want_code)
            assert mx == want_max
            # and the compressor's own stage agrees
            assert np.array_equal(got_len, comp_len)
            assert np.array_equal(got_code, comp_code)
            assert mx == comp_max
    ctx.close()


def test_codebook_noalloc_allocates_nothing(gb):
    """After a warm call, further calls leave the free device memory as it was."""
    rng = np.random.default_rng(23)
    hist = rng.integers(0, 1000, 4096).astype(np.int32)
    h = torch.from_numpy(hist).cuda()
    outs = [gb.codebook_noalloc(h) for _ in range(2)]  # outputs allocated by torch, kept alive
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        gb.codebook_noalloc(h, out=outs[0])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    want_len, _ = ref.huffman_lengths(hist.astype(np.uint32))
    assert np.array_equal(outs[0][0].cpu().numpy(), want_len)


def test_codebook_noalloc_rejects_bad_input(gb):
    z = torch.zeros(1024, dtype=torch.int32, device="cuda")
    with pytest.raises(gb.GbszError):
        gb.codebook_noalloc(z)
    # frequencies whose total reaches 2^32 (two bins of 3e9) are refused
    big = np.zeros(1024, dtype=np.uint32)
    big[3] = big[700] = 3_000_000_000
    hb = torch.from_numpy(big.view(np.int32)).cuda()
    with pytest.raises(gb.GbszError):
        gb.codebook_noalloc(hb)
