"""Corrupt archives on the GPU: every decoder path reports ERR_CORRUPT (or,
for a change that happens to decode, the same status and floats as the
oracle) without a fault, and the context keeps working afterwards.  The
corruptions are built on the CPU from valid archives; every one of them is
caught by a host or kernel check before any access outside the archive."""
import numpy as np
import pytest
import torch

from oracle import ref
from paper_2007_09625_gb300 import workloads

pytestmark = pytest.mark.gpu

CASES = [
    # kind, shape, eb, mode, R, C: 1D through the table decoder (short codes)
    # with one and several tiles per chunk, 1D through the long-code decoder,
    # 2D and 3D; every case has outliers and most have exceptions
    ("walk", (70001,), 1e-4, ref.EB_REL, 16, 256),
    ("walk", (300007,), 1e-4, ref.EB_REL, 512, 2048),
    ("walk", (70001,), 3e-5, ref.EB_REL, 32, 8192),
    ("walk", (50000,), 1e-6, ref.EB_REL, 32768, 1024),
    ("grf", (150, 170), 1e-5, ref.EB_REL, 64, 4096),
    ("lognormal", (21, 23, 25), 1e-4, ref.EB_REL, 64, 128),
    # wide codebooks: codes of 13-16 bits (the general decoder's second table
    # level) and longer (its per-length search) -- 157 + 44 and 520 + 51 of
    # them in the bit-flip test's archives; the targeted test's lognormal
    # archive tops out at 15 bits and so takes the fast decoder instead
    ("grf", (300, 410), 1e-4, ref.EB_REL, 512, 256),
    ("lognormal", (60, 61, 63), 1e-4, ref.EB_REL, 512, 256),
]


@pytest.fixture(scope="module")
def ctx(gb):
    c = gb.Context(0)
    yield c
    c.close()


@pytest.fixture(params=[0, 1, 2, 3], ids=["default", "thread", "warp", "thread-codes"])
def decoder(request):
    return request.param


def gpu_status(gb, ctx, a, shape, decoder=0):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    ctx.set_option(gb.OPT_DECODER, decoder)
    try:
        st = ctx.decompress_status(t, a.size, out)
        torch.cuda.synchronize()
    finally:
        ctx.set_option(gb.OPT_DECODER, 0)
    return st, out.cpu().numpy()


def targeted(a):
    """Changes every decoder must reject."""
    s = ref.sections(a)
    out = {}
    b = a.copy()  # chunk table no longer adds up to the stream length
    o = s["off_bits"]
    v = int.from_bytes(b[o:o + 4].tobytes(), "little") + 1
    b[o:o + 4] = np.frombuffer(v.to_bytes(4, "little"), np.uint8)
    out["bits+1"] = b
    if s["m"] >= 2:
        b = a.copy()  # two outliers out of order
        o = s["off_out"]
        e0, e1 = b[o:o + 8].copy(), b[o + 8:o + 16].copy()
        b[o:o + 8], b[o + 8:o + 16] = e1, e0
        out["outliers_swapped"] = b
    if s["m"] >= 1:
        b = a.copy()  # outlier index past the field
        o = s["off_out"] + 8 * (s["m"] - 1)
        b[o:o + 4] = np.frombuffer(np.uint32(0xFFFFFFF0).tobytes(), np.uint8)
        out["outlier_out_of_range"] = b
    b = a.copy()  # a used symbol loses its code
    used = np.flatnonzero(s["len"])
    b[s["off_len"] + int(used[len(used) // 2])] = 0
    out["length_removed"] = b
    b = a.copy()  # every code one bit longer: Kraft sum below 1 and maxlen changes
    ln = b[s["off_len"]:s["off_len"] + 2 * s["radius"]]
    ln[ln > 0] += 1
    out["lengths_plus_one"] = b
    out["truncated"] = a[:-16].copy()
    for c in sorted({0, s["nanchor"] // 2, s["nanchor"] - 1}) if s["nanchor"] else ():
        b = a.copy()  # a chunk anchor off by one
        o = s["off_anc"] + 4 * c
        b[o:o + 4] = (s["anchors"][c:c + 1] + np.uint32(1)).view(np.uint8)
        out[f"anchor{c}+1"] = b
    return out


@pytest.mark.parametrize("kind,shape,eb,mode,R,C", CASES, ids=[f"{c[0]}{'x'.join(map(str, c[1]))}-R{c[4]}" for c in CASES])
def test_targeted_corruptions_are_rejected(gb, ctx, decoder, kind, shape, eb, mode, R, C):
    x = workloads.field_for(kind, shape, seed=77 + R)
    a = ref.compress(x, eb, mode, radius=R, chunk=C)
    for name, b in targeted(a).items():
        st, _ = gpu_status(gb, ctx, b, shape, decoder)
        assert st != gb.OK, name
        assert ref.decompress_status(b) != ref.OK, name
    # the context still decodes a valid archive
    st, y = gpu_status(gb, ctx, a, shape, decoder)
    assert st == gb.OK and np.array_equal(y.view(np.uint32), ref.decompress(a).view(np.uint32))


@pytest.mark.parametrize("kind,shape,eb,mode,R,C", CASES, ids=[f"{c[0]}{'x'.join(map(str, c[1]))}-R{c[4]}" for c in CASES])
def test_stream_bit_flips_agree_with_oracle(gb, ctx, decoder, kind, shape, eb, mode, R, C):
    """Single-bit flips inside the bitstream: the GPU either rejects the
    archive or decodes it to exactly the oracle's floats."""
    x = workloads.field_for(kind, shape, seed=91 + R)
    a = ref.compress(x, eb, mode, radius=R, chunk=C)
    s = ref.sections(a)
    rng = np.random.default_rng(R + C)
    lo, hi = s["off_str"], a.size
    if s["nanchor"]:  # the anchors too
        lo = s["off_anc"]
    for _ in range(24):
        b = a.copy()
        pos = int(rng.integers(lo, hi))
        b[pos] ^= np.uint8(1 << int(rng.integers(0, 8)))
        st, y = gpu_status(gb, ctx, b, shape, decoder)
        ost = ref.decompress_status(b)
        assert st in (gb.OK, gb.ERR_CORRUPT)
        if st == gb.OK:
            assert ost == ref.OK
            assert np.array_equal(y.view(np.uint32), ref.decompress(b).view(np.uint32))
    st, y = gpu_status(gb, ctx, a, shape, decoder)
    assert st == gb.OK
