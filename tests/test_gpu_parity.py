"""GPU vs oracle parity, stage by stage, through the C ABI.

Tolerance: the whole path is integer and bit-exact, so every stage is
compared for equality -- error-bound scalars, quant codes, histogram, code
lengths, codewords, chunk bit counts, outliers, exceptions, bitstream, the
archive bytes, and the reconstructed floats (0 ulp).  Inputs are seeded
synthetic fields at sizes that span several tiles and a ragged tail.
"""
import numpy as np
import pytest
import torch

from oracle import ref
from paper_2007_09625_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gb):
    c = gb.Context(0)
    yield c
    c.close()


def fold3(x):
    """A 4D field as the 3D field its predictor sees (two slowest axes folded)."""
    return x.reshape((x.shape[0] * x.shape[1],) + x.shape[2:]) if x.ndim == 4 else x


def compare_stages(gb, ctx, x, eb, eb_mode, R, C, lblock=0, order=1):
    """Compress on the GPU and with the oracle; assert each stage equal.
    Returns (gpu archive tensor, nbytes, oracle archive)."""
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    arc, nb = ctx.compress(xt, eb, eb_mode, R, C, lblock=lblock, order=order)
    torch.cuda.synchronize()
    ga = arc[:nb].cpu().numpy()
    n = x.size
    sc = ref.error_bound(x, eb, eb_mode)
    gsc = ctx.debug_copy(gb.DEBUG_SCALARS, 3, np.float32)
    assert np.array_equal(gsc.view(np.uint32), sc.view(np.uint32)), (gsc, sc)
    dq = ref.dualquant(fold3(x), sc, R, lblock=lblock, order=order)
    gcodes = ctx.debug_copy(gb.DEBUG_CODES, n, np.uint16)
    if not np.array_equal(gcodes, dq["codes"]):
        bad = np.flatnonzero(gcodes != dq["codes"])
        raise AssertionError(f"codes differ at {bad.size} points, first {bad[:8]}: "
                             f"gpu {gcodes[bad[:8]]} oracle {dq['codes'][bad[:8]]}")
    hist = ref.histogram(dq["codes"], 2 * R)
    ghist = ctx.debug_copy(gb.DEBUG_HIST, 2 * R, np.uint32)
    assert np.array_equal(ghist, hist)
    ln, mx = ref.huffman_lengths(hist)
    cw = ref.canonical_codes(ln)
    gcw = ctx.debug_copy(gb.DEBUG_CODEWORDS, 2 * R, np.uint64)
    gs = ref.sections(ga)
    assert np.array_equal(gs["len"], ln), "code lengths differ"
    assert np.array_equal(gcw, cw), "canonical codewords differ"
    oa = ref.compress(x, eb, eb_mode, radius=R, chunk=C, lblock=lblock, order=order)
    os_ = ref.sections(oa)
    for key in ("maxlen", "m", "e", "words", "nchunk"):
        assert gs[key] == os_[key], (key, gs[key], os_[key])
    assert np.array_equal(gs["bits"], os_["bits"]), "chunk bit counts differ"
    assert np.array_equal(gs["out_idx"], os_["out_idx"]) and np.array_equal(gs["out_delta"], os_["out_delta"])
    assert np.array_equal(gs["exc_idx"], os_["exc_idx"]) and np.array_equal(gs["exc_raw"], os_["exc_raw"])
    if not np.array_equal(gs["stream"], os_["stream"]):
        bad = np.flatnonzero(gs["stream"] != os_["stream"])
        raise AssertionError(f"bitstream differs in {bad.size} words, first {bad[:8]}")
    assert nb == oa.size and np.array_equal(ga, oa), "archive bytes differ"
    return arc, nb, oa


def decompress_with(gb, ctx, arc, nb, decoder):
    ctx.set_option(gb.OPT_DECODER, decoder)
    try:
        y = ctx.decompress(arc, nb)
        torch.cuda.synchronize()
    finally:
        ctx.set_option(gb.OPT_DECODER, 0)
    return y.cpu().numpy()


def check_decompress(gb, ctx, arc, nb, oa, x, eb, eb_mode):
    """Every decoder (default, thread per chunk, warp per chunk, thread per
    chunk with the codes written out) gives the oracle's floats; those that
    leave decoded codes give the oracle's codes."""
    yo = ref.decompress(oa)
    s_ = ref.sections(oa)
    want_codes = ref.dualquant(fold3(x), ref.error_bound(x, eb, eb_mode), s_["radius"],
                               lblock=s_["lblock"], order=s_["order"])["codes"]
    codes_checked = 0
    for decoder in (0, 1, 2, 3):
        y = decompress_with(gb, ctx, arc, nb, decoder)
        assert y.shape == x.shape
        if not np.array_equal(y.view(np.uint32), yo.view(np.uint32)):
            bad = np.flatnonzero(y.view(np.uint32).ravel() != yo.view(np.uint32).ravel())
            raise AssertionError(f"decoder {decoder}: reconstruction differs at {bad.size} points, first {bad[:8]}")
        try:
            dcodes = ctx.debug_copy(gb.DEBUG_DECODED, x.size, np.uint16)
        except gb.GbszError:  # the fused 1D decoder keeps its codes on chip
            continue
        assert np.array_equal(dcodes, want_codes), decoder
        codes_checked += 1
    assert codes_checked >= 1
    sc = ref.error_bound(x, eb, eb_mode)
    fin = np.isfinite(x)
    err = np.abs(x[fin].astype(np.float64) - y[fin].astype(np.float64))
    assert err.size == 0 or err.max() <= float(sc[0])
    assert np.array_equal(x[~fin].view(np.uint32), y[~fin].view(np.uint32))


CASES = [
    # kind, shape (numpy order), eb, mode, R, C
    ("walk", (100003,), 1e-4, ref.EB_REL, 512, 4096),
    ("walk", (100003,), 1e-4, ref.EB_REL, 512, 64),
    ("walk", (100003,), 1e-4, ref.EB_REL, 512, 8192),
    ("walk", (9000,), 1e-5, ref.EB_REL, 512, 65536),
    ("sinus", (181, 1037), 1e-4, ref.EB_REL, 512, 1024),
    ("grf", (181, 1037), 1e-3, ref.EB_REL, 512, 4096),
    ("grf", (600, 700), 1e-4, ref.EB_REL, 32768, 4096),
    ("sinus", (37, 41, 67), 1e-4, ref.EB_REL, 512, 4096),
    ("lognormal", (37, 41, 67), 1e-3, ref.EB_REL, 512, 256),
    ("lognormal", (40, 40, 40), 1e-5, ref.EB_REL, 32768, 4096),
    ("sinus", (64, 64, 64), 1e-4, ref.EB_REL, 512, 4096),
]


@pytest.mark.parametrize("kind,shape,eb,mode,R,C", CASES, ids=[f"{c[0]}{'x'.join(map(str, c[1]))}-eb{c[2]}-R{c[4]}-C{c[5]}" for c in CASES])
def test_parity(gb, ctx, kind, shape, eb, mode, R, C):
    x = workloads.field_for(kind, shape, seed=sum(shape) + R + C)
    arc, nb, oa = compare_stages(gb, ctx, x, eb, mode, R, C)
    check_decompress(gb, ctx, arc, nb, oa, x, eb, mode)


# 1D fields whose archives carry chunk anchors (chunks of >= 1024 symbols):
# the thread-per-chunk decoder rebuilds each chunk from its anchor.  Several
# thousand chunks (the default decoder is the thread one), ragged last chunks,
# radius 2 (most points outliers), radius 32768 (codes too long for the
# complete table: the general decoder and the separate value pass), chunk
# 65536 (one partial chunk per warp), and non-finite values (exceptions),
# some right before a chunk.
ANCHORED = [
    # n, eb, R, C
    ((1 << 23) + 12345, 1e-4, 512, 1024),
    ((1 << 22) + 777, 1e-4, 512, 2048),
    ((1 << 22) + 5, 1e-4, 2, 1024),
    (3_000_017, 1e-4, 512, 4096),
    (1_000_003, 1e-6, 32768, 1024),
    (300_001, 1e-4, 512, 65536),
]


@pytest.mark.parametrize("n,eb,R,C", ANCHORED, ids=[f"n{c[0]}-R{c[2]}-C{c[3]}" for c in ANCHORED])
def test_parity_anchored_1d(gb, ctx, n, eb, R, C):
    x = workloads.random_walk_1d(n, seed=n % 1000 + C)
    rng = np.random.default_rng(n)
    bad = rng.choice(n, 40, replace=False)
    x[bad[:10]] = np.nan
    x[bad[10:15]] = np.inf
    x[bad[15:20]] = -np.inf
    for c in (1, 2, (n - 1) // C):  # points right before chunks
        if 0 < c * C - 1 < n:
            x[c * C - 1] = np.nan if c % 2 else -np.inf
    arc, nb, oa = compare_stages(gb, ctx, x, eb, ref.EB_REL, R, C)
    s_ = ref.sections(oa)
    assert s_["nanchor"] == (n + C - 1) // C and s_["e"] >= 20
    check_decompress(gb, ctx, arc, nb, oa, x, eb, ref.EB_REL)


EDGE = {
    "n1": np.array([3.25], np.float32),
    "n2": np.array([3.25, -1.0], np.float32),
    "tiny_1d": np.linspace(-1, 1, 37).astype(np.float32),
    "tiny_2d": np.arange(6, dtype=np.float32).reshape(2, 3),
    "tiny_3d": np.random.default_rng(0).normal(size=(2, 3, 5)).astype(np.float32),
    "thin_3d": np.random.default_rng(1).normal(size=(70, 1, 33)).astype(np.float32),
    "col_2d": np.random.default_rng(2).normal(size=(3000, 1)).astype(np.float32),
    "constant_2d": np.full((50, 70), 7.5, np.float32),
    "zeros_3d": np.zeros((9, 10, 11), np.float32),
    "nonfinite": np.where(np.random.default_rng(3).random(5000) < 0.05, np.nan,
                          np.cumsum(np.random.default_rng(4).normal(size=5000))).astype(np.float32),
    "inf_and_huge": np.concatenate([np.cumsum(np.random.default_rng(5).normal(size=3000)),
                                    [np.inf, -np.inf, 3e38, -3e38, 1e-45]]).astype(np.float32),
    "noise_all_outliers": np.random.default_rng(6).normal(size=(20, 30, 40)).astype(np.float32),
}


@pytest.mark.parametrize("name", sorted(EDGE))
@pytest.mark.parametrize("R", [2, 512])
def test_edge_cases(gb, ctx, name, R):
    x = EDGE[name]
    eb, mode = (1e-6, ref.EB_REL) if name == "noise_all_outliers" else (1e-3, ref.EB_REL)
    arc, nb, oa = compare_stages(gb, ctx, x, eb, mode, R, 64)
    check_decompress(gb, ctx, arc, nb, oa, x, eb, mode)


def test_absolute_eb_mode(gb, ctx):
    x = workloads.field_for("grf", (90, 130), seed=7) * np.float32(100)
    arc, nb, oa = compare_stages(gb, ctx, x, 0.05, ref.EB_ABS, 512, 512)
    check_decompress(gb, ctx, arc, nb, oa, x, 0.05, ref.EB_ABS)


def test_determinism_and_repeat_calls(gb, ctx):
    x = workloads.field_for("walk", (50000,), seed=9)
    xt = torch.from_numpy(x).cuda()
    a1, n1 = ctx.compress(xt, 1e-4)
    b1 = a1[:n1].cpu().numpy()
    for _ in range(3):
        a2, n2 = ctx.compress(xt, 1e-4)
        assert n2 == n1 and np.array_equal(a2[:n2].cpu().numpy(), b1)


def test_capacity_error_reports_needed_size(gb, ctx):
    x = workloads.field_for("walk", (20000,), seed=11)
    xt = torch.from_numpy(x).cuda()
    arc, nb = ctx.compress(xt, 1e-4)
    small = torch.empty(nb - 16, dtype=torch.uint8, device="cuda")
    p = gb.make_params([x.size], 1e-4, gb.EB_REL, 512, 0)
    st, need = ctx.compress_status(xt, p, small)
    assert st == gb.ERR_CAPACITY and need == nb
    out = torch.empty(x.size - 1, dtype=torch.float32, device="cuda")
    assert ctx.decompress_status(arc, nb, out) == gb.ERR_CAPACITY


def test_decompress_of_own_archive_checks_the_cached_header(gb, ctx):
    """A decompress of the buffer this context just compressed into plans from
    the header that compress copied back, checked on the device before any
    decoding.  An archive written into the buffer by other means is noticed
    (on the host when the cached plan does not fit the call, else by the
    device check) and decoded from its own header; a change that leaves the
    header alone gives exactly what a decompress reading the header gives."""
    xa = workloads.field_for("walk", (300007,), seed=31)
    xb = workloads.field_for("sinus", (50, 60), seed=32)
    ta, tb = torch.from_numpy(xa).cuda(), torch.from_numpy(xb).cuda()
    arc_b, nb_b = ctx.compress(tb, 1e-4)
    b_bytes = arc_b[:nb_b].clone()
    yb = ref.decompress(ref.compress(xb, 1e-4, ref.EB_REL, 512, gb.auto_chunk(list(xb.shape)[::-1])))
    buf, nba = ctx.compress(ta, 1e-4)
    assert nb_b < nba
    # the smaller archive B in A's buffer, output sized for B (host check)
    buf[:nb_b].copy_(b_bytes)
    out = torch.empty(xb.shape, dtype=torch.float32, device="cuda")
    assert ctx.decompress_status(buf, nba, out) == gb.OK
    assert np.array_equal(out.cpu().numpy().view(np.uint32), yb.view(np.uint32))
    # again with an output large enough for A (the device check)
    buf, nba = ctx.compress(ta, 1e-4, out=buf)
    buf[:nb_b].copy_(b_bytes)
    big = torch.empty(xa.size, dtype=torch.float32, device="cuda")
    assert ctx.decompress_status(buf, nba, big) == gb.OK
    assert np.array_equal(big[:xb.size].cpu().numpy().view(np.uint32), yb.ravel().view(np.uint32))
    # a payload byte changed, header intact: the cached plan against a fresh read
    buf, nba = ctx.compress(ta, 1e-4, out=buf)
    buf[nba - 5] ^= 0x5A
    y1 = torch.empty(xa.size, dtype=torch.float32, device="cuda")
    s1 = ctx.decompress_status(buf, nba, y1)
    ctx.compress(tb, 1e-4)  # the context's cached header now belongs to another buffer
    y2 = torch.empty(xa.size, dtype=torch.float32, device="cuda")
    s2 = ctx.decompress_status(buf, nba, y2)
    assert s1 == s2
    if s1 == gb.OK:
        assert np.array_equal(y1.cpu().numpy().view(np.uint32), y2.cpu().numpy().view(np.uint32))


def test_host_buffer_api(gb, ctx):
    x = workloads.field_for("sinus", (33, 45, 29), seed=12)
    a, nb = ctx.compress_host(x, 1e-4)
    oa = ref.compress(x, 1e-4, ref.EB_REL, 512, gb.auto_chunk(list(x.shape)[::-1]))
    assert nb == oa.size and np.array_equal(a[:nb], oa)
    y = np.empty_like(x)
    ctx.decompress_host(a[:nb], nb, y)
    assert np.array_equal(y.view(np.uint32), ref.decompress(oa).view(np.uint32))


def test_async_host_decompress_pipeline(gb, ctx):
    """gbsz_decompress_host_async: results equal the oracle's while
    synchronous calls run on the context meanwhile; one call may be pending;
    device-side corruption is reported by the wait."""
    xs = [workloads.field_for("walk", (200003,), seed=40 + i) for i in range(3)]
    arcs = [torch.empty(gb.compress_bound([x.size], 1e-4), dtype=torch.uint8).pin_memory() for x in xs]
    outs = [torch.empty(x.shape, dtype=torch.float32).pin_memory() for x in xs]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    nbs = []
    for i, x in enumerate(xs):
        _, nb = ctx.compress_host(torch.from_numpy(x).pin_memory(), 1e-4, out=arcs[i], stream=s1)
        nbs.append(nb)
        ctx.async_wait()
        ctx.decompress_host_async(arcs[i], nb, outs[i], stream=s2)
        if i == 1:
            with pytest.raises(gb.GbszError):  # one pending call at a time
                ctx.decompress_host_async(arcs[0], nbs[0], outs[0], stream=s2)
    ctx.async_wait()
    ctx.async_wait()  # nothing pending: ok
    for i, x in enumerate(xs):
        oa = arcs[i][:nbs[i]].numpy()
        assert np.array_equal(oa, ref.compress(x, 1e-4, ref.EB_REL, 512, gb.auto_chunk([x.size])))
        assert np.array_equal(outs[i].numpy().view(np.uint32), ref.decompress(oa).view(np.uint32)), i
    # chunk 0 claims two more words than it has: the word-offset scan on the
    # device finds the total off, and the wait reports it
    bad = arcs[0][:nbs[0]].clone().pin_memory()
    o = ref.sections(bad.numpy())["off_bits"]
    b0 = int(bad[o:o + 4].numpy().view(np.uint32)[0]) + 64
    bad[o:o + 4] = torch.from_numpy(np.array([b0], np.uint32).view(np.uint8))
    ctx.decompress_host_async(bad, nbs[0], outs[0], stream=s2)
    with pytest.raises(gb.GbszError) as e:
        ctx.async_wait()
    assert e.value.status == gb.ERR_CORRUPT


def test_gpu_decodes_oracle_archives(gb, ctx):
    x = workloads.field_for("lognormal", (21, 30, 50), seed=13)
    oa = ref.compress(x, 1e-4, ref.EB_REL, radius=1024, chunk=128)
    at = torch.from_numpy(oa).cuda()
    y = ctx.decompress(at, oa.size).cpu().numpy()
    assert np.array_equal(y.view(np.uint32), ref.decompress(oa).view(np.uint32))


def fibonacci_walk(levels, seed):
    """1D integer-valued walk whose Lorenzo residuals take `levels` distinct
    values with Fibonacci counts 1, 1, 2, 3, 5, ...: the Huffman tree is a
    chain, so the longest code has levels - 1 bits.  With absolute eb 0.5
    (2eb = 1) every value is its own prequantized integer.  The most frequent
    residual is 0; the others are +-1, +-2, ... with signs chosen (largest
    count first) to keep the drift of the walk small, so every value stays an
    exact float32 integer."""
    F = [1, 1]
    while len(F) < levels:
        F.append(F[-1] + F[-2])
    counts = F[:levels][::-1]  # largest first
    vals, drift = [0], 0
    for k in range(1, levels, 2):
        m = (k + 1) // 2
        ca = counts[k]
        cb = counts[k + 1] if k + 1 < levels else 0
        s = 1 if abs(drift + m * (ca - cb)) <= abs(drift - m * (ca - cb)) else -1
        vals += [s * m, -s * m][: levels - k]
        drift += s * m * (ca - cb)
    rng = np.random.default_rng(seed)
    v = np.repeat(np.array(vals, np.int64), counts)
    rng.shuffle(v)
    x = np.cumsum(v)
    assert np.abs(x).max() < 2 ** 24
    return x.astype(np.float32)


@pytest.mark.parametrize("levels,C", [(12, 64), (16, 4096), (17, 256), (22, 1024), (27, 8192)])
def test_long_codes(gb, ctx, levels, C):
    """Code lengths up to and past the decoder's complete table (15 bits),
    past the encoder's 24-bit codeword form, through both 1D tile-sum paths."""
    x = fibonacci_walk(levels, seed=levels)
    arc, nb, oa = compare_stages(gb, ctx, x, 0.5, ref.EB_ABS, 512, C)
    assert ref.sections(oa)["maxlen"] == levels - 1
    check_decompress(gb, ctx, arc, nb, oa, x, 0.5, ref.EB_ABS)


def test_codes_longer_than_a_word(gb, ctx):
    """A 34-bit longest code (24M symbols): codewords that span two stream
    words and a decoder window that advances twice for one code."""
    x = fibonacci_walk(35, seed=35)
    arc, nb, oa = compare_stages(gb, ctx, x, 0.5, ref.EB_ABS, 512, 4096)
    assert ref.sections(oa)["maxlen"] == 34
    check_decompress(gb, ctx, arc, nb, oa, x, 0.5, ref.EB_ABS)


BLOCK_CASES = [
    # the paper's per-block Lorenzo (Sec. 3.1.1): 32 / 16x16 / 8x8x8 blocks with zero padding
    ("walk", (100003,), 1e-4, ref.EB_REL, 512, 4096),
    ("walk", (70001,), 1e-4, ref.EB_REL, 16, 1024),
    ("sinus", (181, 1037), 1e-4, ref.EB_REL, 512, 1024),
    ("grf", (150, 170), 1e-5, ref.EB_REL, 64, 256),
    ("lognormal", (37, 41, 67), 1e-3, ref.EB_REL, 512, 256),
    ("sinus", (20, 9, 33), 1e-4, ref.EB_REL, 64, 64),
]


@pytest.mark.parametrize("kind,shape,eb,mode,R,C", BLOCK_CASES,
                         ids=[f"blk-{c[0]}{'x'.join(map(str, c[1]))}-R{c[4]}" for c in BLOCK_CASES])
def test_parity_per_block_lorenzo(gb, ctx, kind, shape, eb, mode, R, C):
    x = workloads.field_for(kind, shape, seed=sum(shape) + 3 * R)
    arc, nb, oa = compare_stages(gb, ctx, x, eb, mode, R, C, lblock=1)
    assert ref.sections(oa)["lblock"] == 1
    check_decompress(gb, ctx, arc, nb, oa, x, eb, mode)


ORDER_CASES = [
    # Lorenzo predictor of order n (Sec. 3.1.2, binomial coefficients)
    ("walk", (100003,), 1e-4, ref.EB_REL, 512, 4096, 2),
    ("walk", (70001,), 1e-3, ref.EB_REL, 64, 256, 3),
    ("sinus", (181, 1037), 1e-4, ref.EB_REL, 512, 1024, 2),
    ("grf", (150, 170), 1e-4, ref.EB_REL, 32768, 256, 3),
    ("lognormal", (37, 41, 67), 1e-3, ref.EB_REL, 512, 256, 2),
    ("sinus", (20, 9, 33), 1e-4, ref.EB_REL, 64, 64, 3),
    ("sinus", (70, 1, 45), 1e-4, ref.EB_REL, 512, 1024, 2),
]


@pytest.mark.parametrize("kind,shape,eb,mode,R,C,order", ORDER_CASES,
                         ids=[f"ord{c[6]}-{c[0]}{'x'.join(map(str, c[1]))}-R{c[4]}" for c in ORDER_CASES])
def test_parity_lorenzo_order(gb, ctx, kind, shape, eb, mode, R, C, order):
    x = workloads.field_for(kind, shape, seed=sum(shape) + 5 * R + order)
    arc, nb, oa = compare_stages(gb, ctx, x, eb, mode, R, C, order=order)
    assert ref.sections(oa)["order"] == order
    check_decompress(gb, ctx, arc, nb, oa, x, eb, mode)


def test_lorenzo_order_nonfinite_and_exceptions(gb, ctx):
    x = workloads.field_for("sinus", (90, 110), seed=17)
    x[3, 4] = np.nan
    x[50, 0] = np.inf
    x[7, 99] = np.float32(3e38)
    for order in (2, 3):
        arc, nb, oa = compare_stages(gb, ctx, x, 1e-4, ref.EB_REL, 512, 512, order=order)
        assert ref.sections(oa)["e"] >= 2  # the NaN and the Inf
        check_decompress(gb, ctx, arc, nb, oa, x, 1e-4, ref.EB_REL)


# 1D order-1 fields of 2^23 points and more: the dual-quant kernel leaves a
# code-0 bitmap and a kernel of its own writes the outlier and exception
# records (pack only packs).  Ragged tails, two and four bitmap words a lane
# (chunk 64, chunk >= 128), units of four rounds (chunk 16384), and radius 2,
# which makes most points outliers.
ZB_CASES = [
    ((1 << 23) + 12345, 1e-4, 512, 2048),
    ((1 << 23) + 77, 1e-4, 512, 64),
    ((1 << 23) + 3, 1e-5, 512, 16384),
    (1 << 23, 1e-3, 2, 128),
]


@pytest.mark.parametrize("n,eb,R,C", ZB_CASES, ids=[f"walk{c[0]}-R{c[2]}-C{c[3]}" for c in ZB_CASES])
def test_parity_outlier_kernel(gb, ctx, n, eb, R, C):
    x = workloads.field_for("walk", (n,), seed=n % 1000 + R + C)
    arc, nb, oa = compare_stages(gb, ctx, x, eb, ref.EB_REL, R, C)
    assert ref.sections(oa)["m"] > 0
    check_decompress(gb, ctx, arc, nb, oa, x, eb, ref.EB_REL)


def test_outlier_kernel_exceptions_and_capacity(gb, ctx):
    x = workloads.field_for("walk", ((1 << 23) + 999,), seed=23)
    pos = np.random.default_rng(24).choice(x.size, 300, replace=False)
    x[pos[:150]] = np.nan
    x[pos[150:]] = np.inf
    x[-1] = -np.inf  # the last point of the ragged tail
    arc, nb, oa = compare_stages(gb, ctx, x, 1e-4, ref.EB_REL, 512, 2048)
    s_ = ref.sections(oa)
    assert s_["e"] >= 301 and s_["m"] > s_["e"]
    check_decompress(gb, ctx, arc, nb, oa, x, 1e-4, ref.EB_REL)
    # too small by one byte (the stream's end), and cut inside the outlier records
    xt = torch.from_numpy(x).cuda()
    p = gb.make_params([x.size], 1e-4, gb.EB_REL, 512, 2048)
    for cap in (nb - 1, nb // 3):
        small = torch.empty(cap, dtype=torch.uint8, device="cuda")
        st, need = ctx.compress_status(xt, p, small)
        assert st == gb.ERR_CAPACITY and need == nb, (cap, st, need)


FOLD_CASES = [
    # 4D fields (QMCPACK-like), predicted as 3D over the folded two slowest axes
    ("sinus", (3, 5, 29, 31), 1e-4, 512, 256, 1),
    ("sinus", (6, 10, 33, 47), 1e-3, 512, 1024, 1),
    ("sinus", (4, 3, 17, 23), 1e-4, 64, 128, 2),
]


@pytest.mark.parametrize("kind,shape,eb,R,C,order", FOLD_CASES,
                         ids=[f"4d-{'x'.join(map(str, c[1]))}-ord{c[5]}" for c in FOLD_CASES])
def test_parity_4d_fields(gb, ctx, kind, shape, eb, R, C, order):
    x = workloads.field_for(kind, shape, seed=sum(shape) + order)
    arc, nb, oa = compare_stages(gb, ctx, x, eb, ref.EB_REL, R, C, order=order)
    s_ = ref.sections(oa)
    assert s_["ndim"] == 4
    check_decompress(gb, ctx, arc, nb, oa, x, eb, ref.EB_REL)


@pytest.mark.parametrize("kind,shape,R,C", [("walk", (100003,), 512, 4096), ("grf", (181, 1037), 512, 1024),
                                             ("grf", (300, 200), 32768, 4096), ("lognormal", (37, 41, 67), 512, 256)])
def test_codeword_width_option_keeps_bytes(gb, ctx, kind, shape, R, C):
    """64-bit codeword entries (the paper's enc.64) give the same archive as
    the adaptive 32-bit choice (Sec. 3.2.2)."""
    x = workloads.field_for(kind, shape, seed=sum(shape) + 11)
    xt = torch.from_numpy(x).cuda()
    a32, n32 = ctx.compress(xt, 1e-4, ref.EB_REL, R, C)
    a32 = a32[:n32].clone()
    ctx.set_option(gb.OPT_CODEWORD_BITS, 64)
    try:
        a64, n64 = ctx.compress(xt, 1e-4, ref.EB_REL, R, C)
    finally:
        ctx.set_option(gb.OPT_CODEWORD_BITS, 0)
    torch.cuda.synchronize()
    assert n64 == n32 and torch.equal(a64[:n64], a32)
    assert np.array_equal(a32.cpu().numpy(), ref.compress(x, 1e-4, ref.EB_REL, radius=R, chunk=C))


def test_anchored_decode_into_16_byte_aligned_output(gb, ctx):
    """The decoder that writes the values stores eight values with one 32-byte
    store when the output is 32-byte aligned, else with two 16-byte stores;
    both give the oracle's floats."""
    n, C = (1 << 22) + 3, 1024
    x = workloads.random_walk_1d(n, seed=77)
    oa = ref.compress(x, 1e-4, ref.EB_REL, 512, C)
    yo = ref.decompress(oa)
    arc = torch.from_numpy(oa).cuda()
    for dec in (1, 3):
        ctx.set_option(gb.OPT_DECODER, dec)
        try:
            for off in (0, 4):  # floats: 0 and 16 bytes past a 256-byte aligned allocation
                buf = torch.full((n + 8,), float("nan"), dtype=torch.float32, device="cuda")
                out = buf[off:off + n]
                assert ctx.decompress_status(arc, oa.size, out) == gb.OK
                torch.cuda.synchronize()
                got = buf.cpu().numpy()
                assert np.array_equal(got[off:off + n].view(np.uint32), yo.view(np.uint32)), (dec, off)
                assert np.isnan(got[:off]).all() and np.isnan(got[off + n:]).all(), (dec, off)
        finally:
            ctx.set_option(gb.OPT_DECODER, 0)


@pytest.mark.parametrize("kind,rel", [("sin", 1e-2), ("ramp", 1e-2)])
def test_anchored_without_outliers_and_tiny_codebooks(gb, ctx, kind, rel):
    """Anchored 1D archives with no outlier at all (the chunk starts come
    from a zeroed table) and with codebooks of 1-3 bit codes (the complete
    table that the decoder copies into shared memory has 2-8 entries),
    through the decoder that writes the values and through the two-kernel
    path."""
    n = (1 << 20) + 17
    t = np.arange(n, dtype=np.float64)
    x = ((np.sin(t * 2e-4) + 0.5 * np.sin(t * 7e-5 + 1.0)) if kind == "sin" else t * 1e-3).astype(np.float32)
    arc, nb, oa = compare_stages(gb, ctx, x, rel, ref.EB_REL, 512, 1024)
    s_ = ref.sections(oa)
    assert s_["m"] == 0 and s_["maxlen"] <= 3 and s_["nanchor"] == (n + 1023) // 1024
    check_decompress(gb, ctx, arc, nb, oa, x, rel, ref.EB_REL)
