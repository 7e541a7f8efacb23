"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: a value
derived by hand from the paper's definitions (tests/golden), a closed form
(the d-dimensional prefix sum inverts the Lorenzo first difference), an
invariant (|d - d'| <= eb, Kraft equality, prefix-freeness, histogram sum),
a special case that reduces to a library routine (np.bincount, np.cumsum), or
brute force on tiny inputs (optimal prefix-code cost by exhaustive search).
"""
import heapq
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import ref

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def f32(v):
    return np.float32(v)


# ---------------------------------------------------------------------------
# S0: error bound relative to the value range (Sec. 3.2.2 footnote)

def test_eb_relative_to_value_range():
    x = np.array([1.0, 3.0, -2.0, np.nan, np.inf, -np.inf], np.float32)
    sc = ref.error_bound(x, 0.1, ref.EB_REL)
    # range over finite values = 3 - (-2) = 5; eb = 0.1 * 5 = 0.5
    assert sc[0] == f32(0.5)
    assert sc[1] == f32(1.0)
    assert sc[2] == f32(1.0)


def test_eb_constant_field_and_abs_mode():
    x = np.full(10, 7.25, np.float32)
    assert ref.error_bound(x, 1e-3, ref.EB_REL)[0] == f32(1e-3)
    assert ref.error_bound(np.full(4, np.nan, np.float32), 0.5, ref.EB_REL)[0] == f32(0.5)
    sc = ref.error_bound(x, 0.25, ref.EB_ABS)
    assert list(sc) == [f32(0.25), f32(0.5), f32(2.0)]


def test_eb_rejects_nonpositive():
    with pytest.raises(ref.OracleError):
        ref.error_bound(np.ones(3, np.float32), 0.0, ref.EB_ABS)
    with pytest.raises(ref.OracleError):
        ref.error_bound(np.ones(3, np.float32), -1.0, ref.EB_ABS)


# ---------------------------------------------------------------------------
# S1: prequantization d° = round(d / 2eb) (Sec. 3.1.2) with a watchdog

def exact_dist(d, r):
    return abs(Fraction(float(d)) - Fraction(float(r)))


def recon(q, ebx2):
    return np.float32(np.float32(ebx2) * np.float32(q))


@pytest.mark.parametrize("eb", [0.05, 1e-4, 0.125, 3.3e-3])
def test_prequant_bound_exhaustive_near_ties(eb):
    """Brute force over floats around several tie points: every accepted
    value is within eb exactly, and q is one of the two nearest integers."""
    sc = ref.error_bound(np.zeros(1, np.float32), eb, ref.EB_ABS)
    ebx2 = sc[1]
    for k in (0, 1, 7, 1000, -3, 123457):
        tie = np.float32((k + 0.5) * float(ebx2))
        base = tie.view(np.int32)
        for off in range(-(1 << 13), 1 << 13, 37):
            b = np.int32(base + off)
            if b < 0 and tie > 0:
                continue
            d = b.view(np.float32)
            q, exc = ref.prequant_one(d, sc)
            assert not exc
            r = recon(q, ebx2)
            assert exact_dist(d, r) <= Fraction(float(sc[0])), (eb, k, off)
            # q is floor or ceil of d/(2eb); the exact bound above decides
            t = Fraction(float(d)) / Fraction(float(ebx2))
            assert abs(t - q) < 1


def test_prequant_power_of_two_closed_form():
    """With 2eb a power of two, d/2eb is exact and q = rint(d/2eb)."""
    rng = np.random.default_rng(5)
    sc = ref.error_bound(np.zeros(1, np.float32), 1 / 16, ref.EB_ABS)  # 2eb = 1/8
    x = rng.normal(0, 100, 2000).astype(np.float32)
    want = np.rint(x.astype(np.float64) * 8).astype(np.int64)
    got = [ref.prequant_one(v, sc)[0] for v in x]
    assert np.array_equal(np.array(got), want)


def test_prequant_nonfinite_and_huge_are_exceptions():
    sc = ref.error_bound(np.zeros(1, np.float32), 1e-3, ref.EB_ABS)
    assert ref.prequant_one(np.float32(np.nan), sc) == (0, True)
    assert ref.prequant_one(np.float32(np.inf), sc) == (0, True)
    q, exc = ref.prequant_one(np.float32(3e38), sc)
    assert exc and q == 1 << 30
    q, exc = ref.prequant_one(np.float32(-3e38), sc)
    assert exc and q == -(1 << 30)


def test_prequant_precision_loss_becomes_exception():
    """Above 2^24 multiples of 2eb, float(q) is inexact; points whose
    reconstruction cannot meet eb must be verbatim exceptions."""
    sc = ref.error_bound(np.zeros(1, np.float32), 0.5, ref.EB_ABS)  # 2eb = 1
    xs = np.arange(1 << 25, (1 << 25) + 64, dtype=np.float64).astype(np.float32)
    for d in xs:
        q, exc = ref.prequant_one(d, sc)
        if not exc:
            assert exact_dist(d, recon(q, sc[1])) <= Fraction(0.5)
    # 2^25 + 1 is not a float; values here are multiples of 4 -> float(q) exact
    sc2 = ref.error_bound(np.zeros(1, np.float32), 1e-3, ref.EB_ABS)
    q, exc = ref.prequant_one(np.float32(1e6), sc2)  # t ~ 5e8 >= 2^24
    assert exc or exact_dist(np.float32(1e6), recon(q, sc2[1])) <= Fraction(float(sc2[0]))


# ---------------------------------------------------------------------------
# S2: Lorenzo predictor (Sec. 3.1.2)

def test_lorenzo_golden_2d():
    g = load("worked_2d.json")
    q = np.array(g["q"], np.int32)
    assert np.array_equal(ref.lorenzo_delta(q), np.array(g["delta"], np.int32))


def test_lorenzo_1d_is_first_difference():
    rng = np.random.default_rng(1)
    q = rng.integers(-1000, 1000, 501).astype(np.int32)
    want = np.diff(np.concatenate([[0], q.astype(np.int64)]))
    assert np.array_equal(ref.lorenzo_delta(q), want.astype(np.int32))


def cumsum_all(delta):
    s = delta.astype(np.int64)
    for ax in range(s.ndim):
        s = np.cumsum(s, axis=ax)
    return ((s + (1 << 31)) % (1 << 32) - (1 << 31)).astype(np.int32)


@pytest.mark.parametrize("shape", [(37,), (5, 7), (9, 1), (1, 13), (3, 4, 5), (6, 1, 2), (2, 9, 3)])
def test_lorenzo_inverted_by_prefix_sum(shape):
    """Closed form: the d-dim inclusive prefix sum inverts the order-1
    Lorenzo residual (the decompression cascade of Algorithm 2)."""
    rng = np.random.default_rng(sum(shape))
    q = rng.integers(-2**31, 2**31, shape, dtype=np.int64).astype(np.int32)
    d = ref.lorenzo_delta(q)
    assert np.array_equal(cumsum_all(d), q)


def test_lorenzo_3d_inclusion_exclusion_small():
    q = np.arange(1, 9, dtype=np.int32).reshape(2, 2, 2) ** 2
    d = ref.lorenzo_delta(q)
    # point (1,1,1): q111 - (q011 + q101 + q110) + (q001 + q010 + q100) - q000
    z, y, x = 1, 1, 1
    v = (q[1, 1, 1] - q[1, 1, 0] - q[1, 0, 1] - q[0, 1, 1] + q[1, 0, 0] + q[0, 1, 0] + q[0, 0, 1]
         - q[0, 0, 0])
    assert d[z, y, x] == v


@pytest.mark.parametrize("order", [1, 2, 3])
@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_lorenzo_unit_weight(order, ndim):
    """Sec. 3.1.2: the coefficients sum to 1, so a constant field is
    predicted exactly away from the zero boundary."""
    shape = (order + 3,) * ndim
    q = np.full(shape, 17, np.int32)
    d = ref.lorenzo_delta(q, order=order)
    inner = d[(slice(order, None),) * ndim]
    assert np.all(inner == 0)


def test_lorenzo_order2_1d_binomial():
    # n = 2: p = 2 d[a-1] - d[a-2]  (binomial coefficients C(2,1)=2, C(2,2)=1)
    q = np.array([3, 7, 20, 2, -9], np.int32)
    d = ref.lorenzo_delta(q, order=2)
    assert d[2] == 20 - (2 * 7 - 3) and d[4] == -9 - (2 * 2 - 20)


# ---------------------------------------------------------------------------
# Golden worked example through every stage

def test_worked_example_1d_all_stages():
    g = load("worked_1d.json")
    x = np.array(g["x"], np.float32)
    sc = ref.error_bound(x, g["eb_abs"], ref.EB_ABS)
    assert sc[2] == f32(g["inv2eb"])
    R = g["radius"]
    dq = ref.dualquant(x, sc, R)
    assert list(dq["q"]) == g["q"]
    assert list(dq["codes"]) == g["codes"]
    assert [[int(i), int(d)] for i, d in zip(dq["out_idx"], dq["out_delta"])] == g["outliers"]
    assert dq["exc_idx"].size == 0
    hist = ref.histogram(dq["codes"], 2 * R)
    assert list(hist) == g["histogram"]
    ln, mx = ref.huffman_lengths(hist)
    assert list(ln) == g["lengths"] and mx == 2
    cw = ref.canonical_codes(ln)
    assert list(cw) == g["codewords"]
    bits, stream = ref.deflate(dq["codes"], g["chunk"], ln, cw)
    assert list(bits) == g["bits"] and list(stream) == g["stream"]
    codes = ref.inflate(stream, bits, x.size, g["chunk"], ln)
    assert list(codes) == g["codes"]
    xr = ref.reconstruct(codes, x.shape, R, dq["out_idx"], dq["out_delta"], dq["exc_idx"],
                         dq["exc_raw"], sc[1])
    want = np.float32(sc[1]) * np.array(g["xr_multiples_of_2eb"], np.float32)
    assert np.array_equal(xr, want)
    # and through the archive
    a = ref.compress(x, g["eb_abs"], ref.EB_ABS, radius=R, chunk=g["chunk"])
    assert np.array_equal(ref.decompress(a), want)


# ---------------------------------------------------------------------------
# S2 postquant invariants

def test_postquant_invariants_and_roundtrip():
    rng = np.random.default_rng(3)
    x = np.cumsum(rng.normal(0, 1, (40, 50)), axis=1).astype(np.float32)
    x[3, 4] = np.nan
    x[10, 10] = np.inf
    x[5, 5] = 1e30  # |d / 2eb| >= 2^30 under an absolute bound
    sc = ref.error_bound(x, 1e-3, ref.EB_ABS)
    R = 8
    dq = ref.dualquant(x, sc, R)
    codes = dq["codes"].reshape(x.shape)
    hist = ref.histogram(dq["codes"], 2 * R)
    assert hist.sum() == x.size
    assert hist[0] == dq["out_idx"].size
    assert np.all(np.diff(dq["out_idx"].astype(np.int64)) > 0)
    assert set(dq["exc_idx"]).issubset(set(dq["out_idx"]))
    assert set(dq["exc_idx"].tolist()) == {3 * 50 + 4, 10 * 50 + 10, 5 * 50 + 5}
    # every in-cap code is delta + R in [1, 2R-1]
    delta = ref.lorenzo_delta(dq["q"].reshape(x.shape)).ravel()
    inc = dq["codes"] != 0
    assert np.array_equal(dq["codes"][inc].astype(np.int64) - R, delta[inc])
    assert np.all(np.abs(delta[inc]) < R)
    # the outlier payload restores the residual exactly -> prefix sum gives q
    d2 = np.where(inc, dq["codes"].astype(np.int64) - R, 0)
    d2[dq["out_idx"]] = dq["out_delta"]
    assert np.array_equal(cumsum_all(d2.reshape(x.shape)).ravel(), dq["q"])


def test_postquant_huge_radius_has_no_outliers():
    rng = np.random.default_rng(4)
    x = rng.normal(0, 1, 3000).astype(np.float32)
    sc = ref.error_bound(x, 1e-2, ref.EB_REL)
    dq = ref.dualquant(x, sc, 32768)
    assert dq["out_idx"].size == 0


def test_constant_field_codes():
    x = np.full((6, 7), 2.5, np.float32)
    sc = ref.error_bound(x, 1e-3, ref.EB_ABS)
    dq = ref.dualquant(x, sc, 512)
    # first point carries q itself (2.5 / 0.002 = 1250 > R -> outlier)
    assert dq["codes"][0] == 0 and list(dq["out_idx"]) == [0] and dq["out_delta"][0] == 1250
    # first row / column: delta 0 after the first point; interior: 0
    assert np.all(dq["codes"][1:] == 512)


# ---------------------------------------------------------------------------
# S3 histogram

def test_histogram_is_bincount():
    rng = np.random.default_rng(6)
    c = rng.integers(0, 1024, 100000).astype(np.uint16)
    assert np.array_equal(ref.histogram(c, 1024), np.bincount(c, minlength=1024))


# ---------------------------------------------------------------------------
# S4 Huffman lengths (Sec. 3.2.2) and canonization (Sec. 3.2.3)

def brute_force_optimal_cost(freqs):
    """Minimum sum f*len over all length vectors obeying Kraft (exhaustive)."""
    k = len(freqs)
    best = None
    for lens in itertools.product(range(1, k), repeat=k):
        if sum(Fraction(1, 2 ** l) for l in lens) <= 1:
            c = sum(f * l for f, l in zip(freqs, lens))
            best = c if best is None or c < best else best
    return best


def heap_huffman_cost(freqs):
    h = list(freqs)
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def kraft(ln):
    return sum(Fraction(1, 2 ** int(l)) for l in ln if l)


@pytest.mark.parametrize("seed", range(12))
def test_huffman_optimal_by_brute_force(seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(2, 7))
    freqs = rng.integers(1, 20, k).tolist()
    hist = np.zeros(16, np.uint32)
    syms = rng.choice(16, k, replace=False)
    hist[syms] = freqs
    ln, mx = ref.huffman_lengths(hist)
    cost = int(sum(int(hist[s]) * int(ln[s]) for s in range(16)))
    assert cost == brute_force_optimal_cost(freqs)
    assert kraft(ln) == 1
    assert np.all((ln > 0) == (hist > 0))


@pytest.mark.parametrize("seed", range(6))
def test_huffman_cost_matches_heap_huffman(seed):
    rng = np.random.default_rng(100 + seed)
    hist = rng.geometric(0.05, 1024).astype(np.uint32)
    hist[rng.random(1024) < 0.3] = 0
    ln, mx = ref.huffman_lengths(hist)
    cost = int(np.sum(hist.astype(np.int64) * ln))
    assert cost == heap_huffman_cost([int(f) for f in hist if f])
    assert kraft(ln) == 1
    assert mx == ln.max()


def test_huffman_tie_rule_prefers_leaves():
    """(frequency, symbol) order with leaves first on ties gives the
    minimum-variance tree: all four lengths 2 (internal-first would give
    1,2,3,3)."""
    hist = np.array([1, 1, 2, 2], np.uint32)
    ln, mx = ref.huffman_lengths(hist)
    assert list(ln) == [2, 2, 2, 2] and mx == 2


def test_huffman_single_symbol_and_fibonacci():
    h = np.zeros(8, np.uint32)
    h[5] = 99
    ln, mx = ref.huffman_lengths(h)
    assert list(ln) == [0, 0, 0, 0, 0, 1, 0, 0] and mx == 1
    fib = [1, 1]
    while len(fib) < 20:
        fib.append(fib[-1] + fib[-2])
    ln, mx = ref.huffman_lengths(np.array(fib, np.uint32))
    # Fibonacci weights give the deepest tree: a caterpillar of depth k-1
    assert mx == 19 and sorted(ln.tolist()) == sorted([19] + list(range(1, 20)))


def test_canonical_textbook_example():
    ln = np.array([1, 2, 3, 3], np.uint8)
    assert list(ref.canonical_codes(ln)) == [0b0, 0b10, 0b110, 0b111]


@pytest.mark.parametrize("seed", range(5))
def test_canonical_prefix_free_ordered_complete(seed):
    rng = np.random.default_rng(seed)
    hist = rng.geometric(0.02, 2048).astype(np.uint32)
    hist[rng.random(2048) < 0.5] = 0
    ln, mx = ref.huffman_lengths(hist)
    cw = ref.canonical_codes(ln)
    used = [(int(ln[s]), s, int(cw[s])) for s in range(2048) if ln[s]]
    used.sort()
    strs = [format(c, "0%db" % l) for l, s, c in used]
    # prefix-free: in sorted string order a prefix would sit right before
    ss = sorted(strs)
    assert all(not ss[i + 1].startswith(ss[i]) for i in range(len(ss) - 1))
    # ordered: codes left-aligned to maxlen increase along (len, sym)
    left = [c << (mx - l) for l, s, c in used]
    assert all(left[i] < left[i + 1] for i in range(len(left) - 1))
    # complete (Kraft = 1): first code all zeros, last code all ones
    assert strs[0] == "0" * len(strs[0]) and strs[-1] == "1" * len(strs[-1])


# ---------------------------------------------------------------------------
# S5 / S7 deflate and inflate (Sec. 3.2.4, 3.3)

@pytest.mark.parametrize("chunk", [64, 256, 4096])
def test_deflate_is_concatenation_and_inflate_inverts(chunk):
    rng = np.random.default_rng(chunk)
    n = 5 * chunk + 17
    codes = np.clip(rng.normal(512, 3, n), 0, 1023).astype(np.uint16)
    hist = ref.histogram(codes, 1024)
    ln, mx = ref.huffman_lengths(hist)
    cw = ref.canonical_codes(ln)
    bits, stream = ref.deflate(codes, chunk, ln, cw)
    nc = (n + chunk - 1) // chunk
    assert bits.size == nc and int(bits.sum()) == int(np.sum(ln[codes].astype(np.int64)))
    # brute force: every chunk's words, as a bit string, equal the
    # concatenated codeword strings followed by zero padding
    w = 0
    for c in range(nc):
        seg = codes[c * chunk:(c + 1) * chunk]
        s = "".join(format(int(cw[v]), "0%db" % int(ln[v])) for v in seg)
        nw = (len(s) + 31) // 32
        got = "".join(format(int(v), "032b") for v in stream[w:w + nw])
        assert got == s + "0" * (32 * nw - len(s))
        w += nw
    assert w == stream.size
    assert np.array_equal(ref.inflate(stream, bits, n, chunk, ln), codes)


def test_inflate_rejects_truncated_and_invalid():
    h = np.zeros(8, np.uint32)
    h[3] = 10
    ln, _ = ref.huffman_lengths(h)  # single symbol: "0"; "1" is not a code
    cw = ref.canonical_codes(ln)
    codes = np.full(10, 3, np.uint16)
    bits, stream = ref.deflate(codes, 64, ln, cw)
    assert np.array_equal(ref.inflate(stream, bits, 10, 64, ln), codes)
    with pytest.raises(ref.OracleError):
        ref.inflate(np.array([0x80000000], np.uint32), bits, 10, 64, ln)
    with pytest.raises(ref.OracleError):
        ref.inflate(stream, np.array([9], np.uint32), 10, 64, ln)


# ---------------------------------------------------------------------------
# Whole archive: bound, determinism, corruption

@pytest.mark.parametrize("shape,eb,R,chunk", [
    ((1,), 1e-3, 512, 64),
    ((1000,), 1e-4, 512, 64),
    ((33, 47), 1e-3, 2, 128),
    ((7, 11, 13), 1e-2, 32768, 256),
    ((64, 3), 1e-5, 512, 65536),
])
def test_archive_roundtrip_error_bound(shape, eb, R, chunk):
    rng = np.random.default_rng(len(shape) * 1000 + R)
    x = (np.cumsum(rng.normal(0, 1, shape), axis=-1) + rng.normal(0, 0.1, shape)).astype(np.float32)
    a = ref.compress(x, eb, ref.EB_REL, radius=R, chunk=chunk)
    y = ref.decompress(a)
    sc = ref.error_bound(x, eb, ref.EB_REL)
    err = np.abs(x.astype(np.float64) - y.astype(np.float64))
    assert np.all(err <= float(sc[0]))
    assert a.size <= ref.compress_bound(shape, eb, ref.EB_REL, R, chunk)
    p, n = ref.archive_info(a)
    assert n == x.size and p.radius == R and p.chunk == chunk


def test_archive_nonfinite_verbatim_and_deterministic():
    rng = np.random.default_rng(8)
    x = rng.normal(0, 1, (20, 30)).astype(np.float32)
    x[0, 0] = np.nan
    x[1, 2] = -np.inf
    x[4, 4] = np.float32(1e37)
    nanbits = np.array([0x7FC01234], np.uint32).view(np.float32)[0]
    x[7, 7] = nanbits
    a = ref.compress(x, 1e-3)
    b = ref.compress(x, 1e-3)
    c = ref.compress(x, 1e-3, omp=True)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    y = ref.decompress(a)
    assert np.array_equal(x.view(np.uint32)[~np.isfinite(x)], y.view(np.uint32)[~np.isfinite(x)])
    assert y.view(np.uint32)[7, 7] == 0x7FC01234
    fin = np.isfinite(x)
    sc = ref.error_bound(x, 1e-3, ref.EB_REL)
    assert np.all(np.abs(x[fin].astype(np.float64) - y[fin]) <= float(sc[0]))


def test_corrupt_archives_report_errors_without_crashing():
    rng = np.random.default_rng(9)
    x = np.cumsum(rng.normal(0, 1, 3000)).astype(np.float32)
    a = ref.compress(x, 1e-4, chunk=256)
    assert ref.decompress_status(a[:100]) == ref.ERR_CORRUPT
    assert ref.decompress_status(a[:-4]) == ref.ERR_CORRUPT
    bad = a.copy()
    bad[0] ^= 1
    assert ref.decompress_status(bad) == ref.ERR_CORRUPT
    for t in range(200):
        bad = a.copy()
        pos = int(rng.integers(128, a.size))
        bad[pos] ^= np.uint8(1 << int(rng.integers(0, 8)))
        st = ref.decompress_status(bad)
        assert st in (ref.OK, ref.ERR_CORRUPT)


# ---------------------------------------------------------------------------
# Per-block Lorenzo (Sec. 3.1.1, chunking with a zero padding layer)

def test_block_extents_follow_the_paper():
    # 32 for 1D, 16x16 for 2D, 8x8x8 for 3D (Sec. 3.1.1)
    assert [ref.lorenzo_block_extent(d) for d in (1, 2, 3)] == [32, 16, 8]


@pytest.mark.parametrize("shape", [(70,), (37, 20), (17, 9, 10), (5, 33), (3, 3, 40)])
def test_block_lorenzo_is_the_global_predictor_of_each_block(shape):
    """Zero padding around every block means each block is predicted as if it
    were a field of its own: cut the field into blocks, run the (separately
    pinned) whole-field predictor on each, and the residuals must agree."""
    rng = np.random.default_rng(sum(shape))
    q = rng.integers(-2**31, 2**31, size=shape, dtype=np.int64).astype(np.int32)
    B = ref.lorenzo_block_extent(len(shape))
    got = ref.lorenzo_delta(q, 1, lblock=1)
    want = np.zeros_like(q)
    import itertools
    for starts in itertools.product(*[range(0, s, B) for s in shape]):
        sl = tuple(slice(a, min(a + B, s)) for a, s in zip(starts, shape))
        want[sl] = ref.lorenzo_delta(np.ascontiguousarray(q[sl]), 1)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("shape", [(32,), (16, 16), (8, 8, 8), (7, 5), (3, 4, 2)])
def test_block_lorenzo_equals_global_inside_one_block(shape):
    rng = np.random.default_rng(7)
    q = rng.integers(-1000, 1000, size=shape).astype(np.int32)
    assert np.array_equal(ref.lorenzo_delta(q, 1, lblock=1), ref.lorenzo_delta(q, 1))


def test_block_lorenzo_constant_field_1d():
    # a constant c: every block restarts from the zero padding, so the
    # residual is c at each block start and 0 elsewhere
    q = np.full(100, 41, np.int32)
    d = ref.lorenzo_delta(q, 1, lblock=1)
    want = np.where(np.arange(100) % 32 == 0, 41, 0).astype(np.int32)
    assert np.array_equal(d, want)


@pytest.mark.parametrize("shape,eb", [((3000,), 1e-3), ((50, 61), 1e-4), ((13, 17, 19), 1e-3)])
def test_block_archive_roundtrip_and_header(shape, eb):
    rng = np.random.default_rng(len(shape))
    x = np.cumsum(rng.normal(0, 1, shape), axis=-1).astype(np.float32)
    a = ref.compress(x, eb, ref.EB_REL, radius=64, chunk=256, lblock=1)
    s = ref.sections(a)
    assert s["lblock"] == 1
    y = ref.decompress(a)
    sc = ref.error_bound(x, eb, ref.EB_REL)
    assert np.all(np.abs(x.astype(np.float64) - y) <= float(sc[0]))
    # the quant codes of the archive are those of the per-block dual-quant
    dq = ref.dualquant(x, sc, 64, lblock=1)
    assert np.array_equal(ref.inflate(s["stream"], s["bits"], x.size, 256, s["len"]), dq["codes"])


def test_block_mode_inside_one_block_changes_only_the_flag():
    rng = np.random.default_rng(3)
    x = rng.normal(0, 1, (16, 16)).astype(np.float32)
    a0 = ref.compress(x, 1e-3, ref.EB_REL, radius=512, chunk=64)
    a1 = ref.compress(x, 1e-3, ref.EB_REL, radius=512, chunk=64, lblock=1)
    diff = np.flatnonzero(a0 != a1)
    assert a0.size == a1.size and np.all((diff >= 108) & (diff < 112))


# ---------------------------------------------------------------------------
# Lorenzo predictor of order n > 1 (Sec. 3.1.2, binomial coefficients)

def cumsum_wrap(a, ax):
    s = np.cumsum(a.astype(np.int64), axis=ax)
    return ((s + (1 << 31)) % (1 << 32) - (1 << 31)).astype(np.int32)


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("shape", [(41,), (9, 13), (5, 7, 6), (1, 11), (4, 1, 9)])
def test_lorenzo_order_n_inverted_by_n_prefix_sums(order, shape):
    """Closed form: the order-n residual is the n-th difference along every
    axis (the binomial coefficients of (1 - shift)^n per axis), so n inclusive
    prefix sums along every axis, modulo 2^32, give the integers back."""
    rng = np.random.default_rng(order * 100 + sum(shape))
    q = rng.integers(-2**31, 2**31, shape, dtype=np.int64).astype(np.int32)
    r = ref.lorenzo_delta(q, order=order)
    for _ in range(order):
        for ax in range(r.ndim):
            r = cumsum_wrap(r, ax)
    assert np.array_equal(r, q)


def test_lorenzo_order2_2d_point_by_hand():
    # n = 2 in 2D: the residual at (y, x) is sum over a, b in 0..2 of
    # C(2,a) C(2,b) (-1)^(a+b) q[y-a, x-b]; written out term by term
    rng = np.random.default_rng(5)
    q = rng.integers(-50, 50, (5, 6)).astype(np.int32)
    d = ref.lorenzo_delta(q, order=2)
    y, x = 3, 4
    want = (q[y, x] - 2 * q[y, x - 1] + q[y, x - 2]
            - 2 * q[y - 1, x] + 4 * q[y - 1, x - 1] - 2 * q[y - 1, x - 2]
            + q[y - 2, x] - 2 * q[y - 2, x - 1] + q[y - 2, x - 2])
    assert d[y, x] == want
    # a point on the first row sees only its own row (zeros outside the field)
    assert d[0, 3] == q[0, 3] - 2 * q[0, 2] + q[0, 1]


def test_lorenzo_order3_kills_quadratics():
    # the third difference of a quadratic vanishes away from the boundary
    t = np.arange(40, dtype=np.int64)
    q = (3 * t * t - 7 * t + 11).astype(np.int32)
    d = ref.lorenzo_delta(q, order=3)
    assert np.all(d[3:] == 0) and np.any(d[:3] != 0)


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("shape", [(50,), (7, 9), (4, 5, 6)])
def test_reconstruct_order_n_recovers_integers(order, shape):
    """The cascading reconstruction (each point predicted from the points
    already rebuilt) inverts the order-n residual: with 2eb = 1 the output is
    the prequantized integers themselves."""
    rng = np.random.default_rng(order + len(shape))
    q = rng.integers(-3000, 3000, shape).astype(np.int32)
    flat = ref.lorenzo_delta(q, order=order).ravel()
    R = 64
    inc = np.abs(flat) < R
    codes = np.where(inc, flat + R, 0).astype(np.uint16)
    oi = np.flatnonzero(~inc).astype(np.uint32)
    e = np.zeros(0, np.uint32)
    x = ref.reconstruct(codes, shape, R, oi, flat[~inc], e, e, 1.0, order=order)
    assert np.array_equal(x, q.astype(np.float32))


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("shape,eb", [((3001,), 1e-3), ((45, 61), 1e-4), ((11, 17, 19), 1e-3)])
def test_order_n_archive_roundtrip_and_codes(order, shape, eb):
    rng = np.random.default_rng(order * 7 + len(shape))
    x = np.cumsum(np.cumsum(rng.normal(0, 1, shape), axis=-1), axis=0).astype(np.float32)
    a = ref.compress(x, eb, ref.EB_REL, radius=128, chunk=256, order=order)
    s = ref.sections(a)
    assert s["order"] == order
    y = ref.decompress(a)
    sc = ref.error_bound(x, eb, ref.EB_REL)
    assert np.all(np.abs(x.astype(np.float64) - y) <= float(sc[0]))
    dq = ref.dualquant(x, sc, 128, order=order)
    assert np.array_equal(ref.inflate(s["stream"], s["bits"], x.size, 256, s["len"]), dq["codes"])


def test_order_defaults_and_limits():
    rng = np.random.default_rng(2)
    x = rng.normal(0, 1, (20, 20)).astype(np.float32)
    a0 = ref.compress(x, 1e-3, order=0)
    a1 = ref.compress(x, 1e-3, order=1)
    assert np.array_equal(a0, a1) and ref.sections(a1)["order"] == 1
    with pytest.raises(ref.OracleError):
        ref.compress(x, 1e-3, order=4)
    with pytest.raises(ref.OracleError):
        ref.compress(x, 1e-3, order=2, lblock=1)


# ---------------------------------------------------------------------------
# 4D fields (QMCPACK-like, 288x115x69x69 in the paper's datasets) are
# predicted as 3D with the two slowest axes folded into one

def test_4d_archive_is_the_folded_3d_archive():
    rng = np.random.default_rng(4)
    x4 = np.cumsum(rng.normal(0, 1, (3, 4, 5, 6)), axis=-1).astype(np.float32)
    a4 = ref.compress(x4, 1e-3, chunk=64)
    a3 = ref.compress(x4.reshape(12, 5, 6), 1e-3, chunk=64)
    diff = set(np.flatnonzero(a4 != a3).tolist())
    header_fields = set(range(8, 12)) | set(range(32, 40)) | set(range(124, 128))  # ndim, dims[2], dims[3]
    assert a4.size == a3.size and diff and diff <= header_fields
    p, n = ref.archive_info(a4)
    assert p.ndim == 4 and [p.dims[i] for i in range(4)] == [6, 5, 4, 3] and n == x4.size
    y = ref.decompress(a4)
    assert y.shape == x4.shape
    sc = ref.error_bound(x4, 1e-3, ref.EB_REL)
    assert np.all(np.abs(x4.astype(np.float64) - y) <= float(sc[0]))


# ---------------------------------------------------------------------------
# Chunk anchors (this format's section): 1D fields, one order-1 predictor,
# chunks of at least 1024 symbols

def _residuals(x, sc, R):
    """Lorenzo residual of every point, from the dual-quant outputs: code - R,
    or the outlier's residual for code 0."""
    dq = ref.dualquant(x, sc, R)
    d = dq["codes"].astype(np.int64) - R
    d[dq["out_idx"]] = dq["out_delta"]
    return d


@pytest.mark.parametrize("n,chunk", [(20000, 1024), (65536, 4096), (9000, 65536), (70001, 2048)])
def test_anchor_is_the_prefix_of_the_residuals(n, chunk):
    """Order-1 1D Lorenzo residuals are first differences of the prequantized
    integers, so the integer of the point before chunk c is the sum of every
    residual before it (mod 2^32); the first chunk's anchor is 0.  The values
    the oracle rebuilds there are fl(2eb * anchor), within eb of the input."""
    rng = np.random.default_rng(n + chunk)
    x = np.cumsum(rng.normal(0, 1e-2, n)).astype(np.float32)
    x[rng.choice(n, n // 100, replace=False)] = rng.uniform(x.min(), x.max(), n // 100).astype(np.float32)
    x[chunk - 1 if chunk < n else 0] = np.nan  # an exception right before a chunk
    R = 512
    a = ref.compress(x, 1e-4, ref.EB_REL, R, chunk)
    s = ref.sections(a)
    nc = (n + chunk - 1) // chunk
    assert s["nanchor"] == nc and s["anchors"].size == nc
    sc = ref.error_bound(x, 1e-4, ref.EB_REL)
    pre = np.concatenate([[0], np.cumsum(_residuals(x, sc, R))]) % (1 << 32)
    want = np.array([pre[c * chunk] for c in range(nc)], np.uint64)
    assert np.array_equal(s["anchors"].astype(np.uint64), want)
    assert s["anchors"][0] == 0
    y = ref.decompress(a)
    for c in range(1, nc):
        p = c * chunk - 1
        if np.isfinite(x[p]):
            qf = np.float32(np.int32(np.uint32(s["anchors"][c])))
            assert (np.float32(sc[1]) * qf).view(np.uint32) == y[p].view(np.uint32)
            assert abs(float(x[p]) - float(y[p])) <= float(sc[0])
        else:  # a non-finite value predicts as the integer 0
            assert s["anchors"][c] == 0


@pytest.mark.parametrize("shape,chunk,lblock,order", [((20000,), 512, 0, 1), ((20000,), 4096, 1, 1),
                                                      ((20000,), 4096, 0, 2), ((100, 200), 4096, 0, 1),
                                                      ((10, 20, 30), 2048, 0, 1)])
def test_no_anchors_outside_their_case(shape, chunk, lblock, order):
    # no section: the outliers follow the chunk table directly
    rng = np.random.default_rng(chunk)
    x = np.cumsum(rng.normal(0, 1, shape), axis=-1).astype(np.float32)
    a = ref.compress(x, 1e-3, ref.EB_REL, 512, chunk, lblock=lblock, order=order)
    s = ref.sections(a)
    assert s["nanchor"] == 0 and s["off_out"] == ((s["off_bits"] + 4 * s["nchunk"] + 15) & ~15)
    assert s["total"] == a.size


def test_corrupt_anchor_is_detected():
    rng = np.random.default_rng(11)
    n, chunk = 30000, 1024
    x = np.cumsum(rng.normal(0, 1e-2, n)).astype(np.float32)
    a = ref.compress(x, 1e-4, ref.EB_REL, 512, chunk)
    s = ref.sections(a)
    assert ref.decompress_status(a) == ref.OK
    for c in (0, 1, s["nchunk"] // 2, s["nchunk"] - 1):
        b = a.copy()
        b[s["off_anc"] + 4 * c] ^= np.uint8(4)
        assert ref.decompress_status(b) == ref.ERR_CORRUPT, c
