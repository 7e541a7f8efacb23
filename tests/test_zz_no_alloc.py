"""gbsz_codebook_noalloc -- the codebook entry point for callers that cannot
allocate device memory (graph capture, caller-owned memory pools, fixed
budgets) -- must give exactly what the compressor's own codebook stage
gives: the same code lengths and canonical codewords for the same histogram
(integer results, compared for equality), on consecutive calls.

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


def test_codebook_noalloc_matches_compressor(gb):
    ctx = gb.Context(0)
    cases = [
        (workloads.field_for("walk", (200003,), seed=21), 1e-4, 512),
        (workloads.field_for("lognormal", (30, 40, 50), seed=22), 1e-5, 32768),
    ]
    for x, rel, R in cases:
        hist, want_len, want_code, want_max = compressor_codebook(gb, ctx, x, rel, R)
        h = torch.from_numpy(hist.view(np.int32)).cuda()
        for _ in range(2):  # consecutive calls share the library's scratch
            ln, code, mx = gb.codebook_noalloc(h)
            torch.cuda.synchronize()
            assert np.array_equal(ln.cpu().numpy(), want_len)
            assert np.array_equal(code.cpu().numpy().view(np.uint64), want_code)
            assert mx == want_max
    ctx.close()


def test_codebook_noalloc_rejects_bad_input(gb):
    z = torch.zeros(1024, dtype=torch.int32, device="cuda")
    with pytest.raises(gb.GbszError):
        gb.codebook_noalloc(z)
