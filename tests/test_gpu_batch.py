"""Batched compress/decompress: every field of a batch gives exactly the
bytes (archive) and floats (reconstruction) that a single-field call gives,
and the oracle too.  Batch compress runs every stage of all fields in one
launch per kernel (grouped) or the fields' own launches on several internal
streams; both are checked, so this also checks that no state leaks between
fields running together."""
import numpy as np
import pytest
import torch

from oracle import ref
from paper_2007_09625_gb300 import workloads

pytestmark = pytest.mark.gpu


def mixed_fields(count, seed):
    rng = np.random.default_rng(seed)
    kinds = [("walk", 1), ("sinus", 2), ("grf", 2), ("lognormal", 3), ("sinus", 3)]
    out = []
    for i in range(count):
        kind, rank = kinds[i % len(kinds)]
        if rank == 1:
            shape = (int(rng.integers(1000, 300000)),)
        elif rank == 2:
            shape = (int(rng.integers(20, 400)), int(rng.integers(20, 700)))
        else:
            shape = tuple(int(v) for v in rng.integers(5, 60, 3))
        if kind == "grf" and rank == 3:
            kind = "lognormal"
        out.append(workloads.field_for(kind, shape, seed=seed + i))
    return out


@pytest.fixture(scope="module")
def ctx(gb):
    c = gb.Context(0)
    yield c
    c.close()


def test_batch_matches_single_calls_and_oracle(gb, ctx):
    fields = mixed_fields(13, seed=300)  # more fields than internal streams
    ebs = [1e-4, 1e-3, 1e-5] * 5
    rads = [512, 512, 32768, 64] * 4
    ts = [torch.from_numpy(f).cuda() for f in fields]
    arcs, nbs, sts = ctx.compress_batch(ts, ebs[:13], gb.EB_REL, rads[:13], 0)
    torch.cuda.synchronize()
    assert all(s == gb.OK for s in sts)
    for i, f in enumerate(fields):
        single, nb1 = ctx.compress(ts[i], ebs[i], gb.EB_REL, rads[i], 0)
        a_b = arcs[i][:nbs[i]].cpu().numpy()
        assert nbs[i] == nb1 and np.array_equal(a_b, single[:nb1].cpu().numpy()), i
        chunk = gb.auto_chunk(list(f.shape)[::-1], rads[i])
        oa = ref.compress(f, ebs[i], ref.EB_REL, rads[i], chunk)
        assert np.array_equal(a_b, oa), i
    outs = [torch.empty_like(t) for t in ts]
    outs, dsts = ctx.decompress_batch(arcs, nbs, outs)
    torch.cuda.synchronize()
    assert all(s == gb.OK for s in dsts)
    for i, f in enumerate(fields):
        yo = ref.decompress(arcs[i][:nbs[i]].cpu().numpy())
        assert np.array_equal(outs[i].cpu().numpy().view(np.uint32), yo.view(np.uint32)), i


def test_batch_reports_per_field_errors(gb, ctx):
    fields = mixed_fields(4, seed=400)
    ts = [torch.from_numpy(f).cuda() for f in fields]
    params = [gb.make_params(gb.field_dims(t), 1e-4) for t in ts]
    outs = [torch.empty(gb.load().gbsz_compress_bound(__import__("ctypes").byref(p)), dtype=torch.uint8,
                        device="cuda") for p in params]
    outs[2] = torch.empty(64, dtype=torch.uint8, device="cuda")  # far too small
    with pytest.raises(gb.GbszError):
        ctx.compress_batch(ts, 1e-4, outs=outs, params=params)
    # the other fields still complete correctly
    import ctypes as C
    k = len(ts)
    P = (gb.Params * k)(*params)
    fp = (C.c_void_p * k)(*[t.data_ptr() for t in ts])
    ap = (C.c_void_p * k)(*[o.data_ptr() for o in outs])
    caps = (C.c_size_t * k)(*[o.numel() for o in outs])
    nb = (C.c_size_t * k)()
    sts = (C.c_int * k)()
    st = gb.load().gbsz_compress_batch(ctx.h, k, fp, P, ap, caps, nb, sts, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == gb.ERR_CAPACITY and list(sts) == [0, 0, gb.ERR_CAPACITY, 0] and nb[2] > 64
    for i in (0, 1, 3):
        single, n1 = ctx.compress(ts[i], 1e-4)
        assert nb[i] == n1 and torch.equal(outs[i][:n1], single[:n1])


def test_batch_graph_replay_follows_new_data(gb, ctx):
    """On a stream of its own, the second identical batch call is captured as
    a CUDA graph and later ones replay it: replays must read the fields'
    current contents, and a changed parameter or header must not replay."""
    s = torch.cuda.Stream()
    fields = mixed_fields(5, seed=600)
    ts = [torch.from_numpy(f).cuda() for f in fields]
    params = [gb.make_params(gb.field_dims(t), 1e-4) for t in ts]
    arcs = [torch.empty(gb.load().gbsz_compress_bound(__import__("ctypes").byref(p)), dtype=torch.uint8,
                        device="cuda") for p in params]
    outs = [torch.empty_like(t) for t in ts]
    torch.cuda.synchronize()

    def run():
        _, nbs, sts = ctx.compress_batch(ts, None, outs=arcs, params=params, stream=s)
        ctx.decompress_batch(arcs, nbs, outs, stream=s)
        s.synchronize()
        return list(nbs)

    def check(nbs):
        for i, f in enumerate(fields):
            oa = ref.compress(f, 1e-4, ref.EB_REL, 512, gb.auto_chunk(list(f.shape)[::-1], 512))
            assert nbs[i] == oa.size and np.array_equal(arcs[i][:nbs[i]].cpu().numpy(), oa), i
            assert np.array_equal(outs[i].cpu().numpy().view(np.uint32), ref.decompress(oa).view(np.uint32)), i

    g0 = ctx.debug_copy(gb.DEBUG_GRAPHS, 4, np.uint64)
    for _ in range(4):  # eager (allocates), eager or captured, then replayed
        check(run())
    g1 = ctx.debug_copy(gb.DEBUG_GRAPHS, 4, np.uint64)
    assert all(int(v) >= 1 for v in g1 - g0), (g0, g1)  # each kind captured and replayed
    # same pointers and parameters, new contents: the replay must see them
    rng = np.random.default_rng(9)
    for i, f in enumerate(fields):
        f += np.float32(0.5) * rng.standard_normal(f.shape).astype(np.float32)
        ts[i].copy_(torch.from_numpy(f))
    torch.cuda.synchronize()
    for _ in range(2):
        check(run())
    # a different parameter is a different batch
    params[2] = gb.make_params(gb.field_dims(ts[2]), 1e-3)
    nbs = run()
    oa = ref.compress(fields[2], 1e-3, ref.EB_REL, 512, gb.auto_chunk(list(fields[2].shape)[::-1], 512))
    assert nbs[2] == oa.size and np.array_equal(arcs[2][:nbs[2]].cpu().numpy(), oa)


def test_autotune_choice_is_remembered_and_reproducible(gb, ctx):
    """The tuner picks one of its candidates, remembers it per (rank, dims,
    radius), and single and batched calls with its parameters give the
    oracle's archive for that chunk."""
    f = workloads.field_for("grf", (300, 700), seed=11)
    t = torch.from_numpy(f).cuda()
    p, ms = ctx.autotune(t, 1e-4)
    assert p.chunk in (256, 512, 1024, 2048, 4096, gb.auto_chunk([700, 300], 512)) and ms > 0
    p2, ms2 = ctx.autotune(t, 1e-4)
    assert p2.chunk == p.chunk and ms2 == 0.0
    arc, nb = ctx.compress_params(t, p)
    oa = ref.compress(f, 1e-4, ref.EB_REL, 512, p.chunk)
    assert nb == oa.size and np.array_equal(arc[:nb].cpu().numpy(), oa)
    arcs, nbs, _ = ctx.compress_batch([t, t], None, params=[p, p])
    torch.cuda.synchronize()
    assert all(n_ == oa.size and np.array_equal(a[:n_].cpu().numpy(), oa) for a, n_ in zip(arcs, nbs))


def test_autotune_reports_knobs_and_tuned_calls_match_oracle(gb, ctx):
    """The tuner's decoder and tile-extent choices are reported per key, and
    compress / decompress calls that use them (options at 0) give the
    oracle's archive and floats."""
    for kind, shape in (("lognormal", (40, 48, 56)), ("grf", (257, 333))):
        f = workloads.field_for(kind, shape, seed=12)
        t = torch.from_numpy(f).cuda()
        p, _ = ctx.autotune(t, 1e-4)
        chunk, decoder, slab = ctx.tuned_knobs(p)
        assert chunk == p.chunk
        assert decoder in ((1, 2) if p.chunk <= 4096 else (0,))
        assert slab in (0, 4, 8, 16, 32, 64)
        arc, nb = ctx.compress_params(t, p)
        oa = ref.compress(f, 1e-4, ref.EB_REL, 512, p.chunk)
        assert nb == oa.size and np.array_equal(arc[:nb].cpu().numpy(), oa)
        y = ctx.decompress(arc, nb)
        torch.cuda.synchronize()
        assert np.array_equal(y.cpu().numpy().view(np.uint32), ref.decompress(oa).view(np.uint32))
    with pytest.raises(gb.GbszError):
        ctx.tuned_knobs(gb.make_params([5, 6, 7], 1e-4))


@pytest.mark.parametrize("kind,shape,lblock", [("lognormal", (37, 41, 67), 0), ("sinus", (45, 50, 61), 1),
                                               ("grf", (181, 1037), 0), ("sinus", (150, 170), 1)])
def test_lorenzo_slab_option_keeps_bytes(gb, ctx, kind, shape, lblock):
    """Any dual-quant tile extent along the swept dimension gives the
    oracle's archive, in single and grouped batch calls."""
    f = workloads.field_for(kind, shape, seed=13)
    t = torch.from_numpy(f).cuda()
    oa = ref.compress(f, 1e-4, ref.EB_REL, 512, 1024, lblock=lblock)
    try:
        for slab in (1, 3, 4, 7, 16, 64, 1000):
            ctx.set_option(gb.OPT_LORENZO_SLAB, slab)
            arc, nb = ctx.compress(t, 1e-4, gb.EB_REL, 512, 1024, lblock=lblock)
            torch.cuda.synchronize()
            assert nb == oa.size and np.array_equal(arc[:nb].cpu().numpy(), oa), slab
            p = gb.make_params(gb.field_dims(t), 1e-4, gb.EB_REL, 512, 1024, lblock=lblock)
            arcs, nbs, _ = ctx.compress_batch([t, t], None, params=[p, p])
            torch.cuda.synchronize()
            assert all(n_ == oa.size and np.array_equal(a[:n_].cpu().numpy(), oa) for a, n_ in zip(arcs, nbs)), slab
    finally:
        ctx.set_option(gb.OPT_LORENZO_SLAB, 0)
    with pytest.raises(gb.GbszError):
        ctx.set_option(gb.OPT_LORENZO_SLAB, 65537)


def test_batch_with_orders_blocks_and_4d(gb, ctx):
    """A batch mixing Lorenzo orders, the per-block mode and a 4D field gives
    each field's single-call archive and the oracle's."""
    shapes = [(60001,), (90, 130), (17, 23, 29), (3, 4, 19, 21), (40000,), (55, 66)]
    fields = [workloads.field_for("walk" if len(s) == 1 else "sinus", s, seed=900 + i) for i, s in enumerate(shapes)]
    opts = [(2, 0), (3, 0), (2, 0), (1, 0), (1, 1), (1, 1)]  # (order, lblock)
    ts = [torch.from_numpy(f).cuda() for f in fields]
    params = [gb.make_params(gb.field_dims(t), 1e-4, gb.EB_REL, 512, 256, lblock=lb, order=o)
              for t, (o, lb) in zip(ts, opts)]
    arcs, nbs, sts = ctx.compress_batch(ts, None, params=params)
    torch.cuda.synchronize()
    assert all(s == gb.OK for s in sts)
    for i, f in enumerate(fields):
        o, lb = opts[i]
        oa = ref.compress(f, 1e-4, ref.EB_REL, 512, 256, lblock=lb, order=o)
        assert np.array_equal(arcs[i][:nbs[i]].cpu().numpy(), oa), i
    outs = [torch.empty_like(t) for t in ts]
    outs, dsts = ctx.decompress_batch(arcs, nbs, outs)
    torch.cuda.synchronize()
    assert all(s == gb.OK for s in dsts)
    for i in range(len(fields)):
        yo = ref.decompress(arcs[i][:nbs[i]].cpu().numpy())
        assert np.array_equal(outs[i].cpu().numpy().view(np.uint32), yo.view(np.uint32)), i


def test_single_calls_replayed_as_graphs_follow_new_data(gb, ctx):
    """Identical single-field calls on a capturable stream are replayed as
    CUDA graphs; a replay reads the buffers' current contents, so new data in
    the same buffers gives that data's archive and reconstruction."""
    s = torch.cuda.Stream()
    x = torch.from_numpy(workloads.field_for("sinus", (90, 130), seed=71)).cuda()
    arc = torch.empty(gb.compress_bound(gb.field_dims(x), 1e-4), dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    g0 = ctx.debug_copy(gb.DEBUG_GRAPHS_SINGLE, 4, np.uint64)
    # the same data four times (each kind: eager, eager, captured, replayed),
    # then new data in the same buffers (the compress graph replays on it)
    for i, seed in enumerate([71, 71, 71, 71, 72, 73]):
        f = workloads.field_for("sinus", (90, 130), seed=seed)
        with torch.cuda.stream(s):
            x.copy_(torch.from_numpy(f))
        s.synchronize()
        _, nb = ctx.compress(x, 1e-4, out=arc, stream=s)
        ctx.decompress(arc, nb, out=y, stream=s)
        s.synchronize()
        oa = ref.compress(f, 1e-4, ref.EB_REL, 512, gb.auto_chunk([130, 90]))
        assert nb == oa.size and np.array_equal(arc[:nb].cpu().numpy(), oa), i
        assert np.array_equal(y.cpu().numpy().view(np.uint32), ref.decompress(oa).view(np.uint32)), i
    g1 = ctx.debug_copy(gb.DEBUG_GRAPHS_SINGLE, 4, np.uint64)
    d = g1 - g0
    assert d[0] >= 1 and d[1] >= 1 and d[2] >= 1 and d[3] >= 1, (g0, g1)


def test_profiling_survives_graph_replay(gb, ctx):
    """Stage timing while identical calls are captured and replayed: every
    call of every stage is counted, with a positive time, and the archive
    and reconstruction stay the oracle's."""
    s = torch.cuda.Stream()
    f = workloads.field_for("walk", (300001,), seed=81)
    x = torch.from_numpy(f).cuda()
    arc = torch.empty(gb.compress_bound(gb.field_dims(x), 1e-4), dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    g0 = ctx.debug_copy(gb.DEBUG_GRAPHS_SINGLE, 4, np.uint64)
    ctx.profile_read()
    ctx.profile_enable(True)
    calls = 6
    try:
        for _ in range(calls):
            _, nb = ctx.compress(x, 1e-4, out=arc, stream=s)
            ctx.decompress(arc, nb, out=y, stream=s)
        s.synchronize()
        ms, cnt, launches = ctx.profile_read()
    finally:
        ctx.profile_enable(False)
    g1 = ctx.debug_copy(gb.DEBUG_GRAPHS_SINGLE, 4, np.uint64)
    assert (g1 - g0)[1] >= 1 and (g1 - g0)[3] >= 1, (g0, g1)  # compress and decompress replayed
    for i, name in enumerate(gb.STAGES[:10]):
        assert cnt[i] == calls and ms[i] > 0, (name, cnt[i], ms[i])
    assert launches > 0
    oa = ref.compress(f, 1e-4, ref.EB_REL, 512, gb.auto_chunk([f.size]))
    assert nb == oa.size and np.array_equal(arc[:nb].cpu().numpy(), oa)
    assert np.array_equal(y.cpu().numpy().view(np.uint32), ref.decompress(oa).view(np.uint32))


def test_grouped_batch_equals_slot_streams_and_oracle(gb, ctx):
    """One launch per stage for the whole batch: ranks 1-4, absolute and
    relative bounds, radii from 64 to 32768, chunks 64 to 8192, the per-block
    mode, a field whose pointer is not 16-byte aligned (and whose 1D archive
    carries chunk anchors); the archives equal the slot-stream path's and the
    oracle's."""
    rng = np.random.default_rng(950)
    kinds = [("walk", (70001,)), ("sinus", (90, 131)), ("lognormal", (17, 23, 29)), ("walk", (1,)),
             ("grf", (200, 300)), ("sinus", (3, 4, 19, 21)), ("walk", (300007,)), ("lognormal", (40, 40, 41))]
    fields, params, ts = [], [], []
    base = torch.empty(400_000, dtype=torch.float32, device="cuda")
    for i, (kind, shape) in enumerate(kinds):
        f = workloads.field_for(kind if len(shape) < 4 else "sinus", shape if len(shape) < 4 else shape[1:],
                                seed=960 + i)
        if len(shape) == 4:
            f = np.concatenate([f[None] * (1 + 0.01 * k) for k in range(shape[0])]).astype(np.float32)
        fields.append(f)
        if i == 6:  # a view 4 bytes into a buffer: not 16-byte aligned
            t = base[1:1 + f.size].view(f.shape)
            t.copy_(torch.from_numpy(f))
        else:
            t = torch.from_numpy(f).cuda()
        ts.append(t)
        mode = gb.EB_ABS if i % 3 == 2 else gb.EB_REL
        eb = 1e-3 if mode == gb.EB_ABS else [1e-4, 1e-3, 1e-2][i % 3]
        R = [512, 64, 32768, 512][i % 4]
        C = [0, 64, 256, 8192][i % 4] if i != 6 else 2048  # field 6: 1D in chunks of 2048, with chunk anchors
        params.append(gb.make_params(gb.field_dims(t), eb, mode, R, C, lblock=1 if i in (1, 4) else 0))
    torch.cuda.synchronize()
    results = {}
    for mode_ in (0, 1):
        ctx.set_option(gb.OPT_BATCH_MODE, mode_)
        try:
            arcs, nbs, sts = ctx.compress_batch(ts, None, params=params)
            torch.cuda.synchronize()
        finally:
            ctx.set_option(gb.OPT_BATCH_MODE, 0)
        assert all(s_ == gb.OK for s_ in sts), sts
        results[mode_] = [a[:n].cpu().numpy() for a, n in zip(arcs, nbs)]
    oas = []
    for i, f in enumerate(fields):
        p = params[i]
        oa = ref.compress(f, p.eb, p.eb_mode, p.radius, p.chunk or gb.auto_chunk(list(f.shape)[::-1], p.radius),
                          lblock=p.lorenzo_block)
        assert np.array_equal(results[0][i], results[1][i]), i
        assert np.array_equal(results[0][i], oa), i
        oas.append(oa)
    # and back, both ways, to the oracle's floats
    arcs = [torch.from_numpy(a).cuda() for a in oas]
    nbs = [a.size for a in oas]
    for mode_ in (0, 1):
        outs = [torch.empty(f.shape, dtype=torch.float32, device="cuda") for f in fields]
        ctx.set_option(gb.OPT_BATCH_MODE, mode_)
        try:
            outs, dsts = ctx.decompress_batch(arcs, nbs, outs)
            torch.cuda.synchronize()
        finally:
            ctx.set_option(gb.OPT_BATCH_MODE, 0)
        assert all(s_ == gb.OK for s_ in dsts), (mode_, dsts)
        for i, oa in enumerate(oas):
            yo = ref.decompress(oa)
            assert np.array_equal(outs[i].cpu().numpy().view(np.uint32), yo.view(np.uint32)), (mode_, i)


def test_grouped_batch_reports_corrupt_fields(gb, ctx):
    """A corrupt archive inside a grouped decompress batch fails alone."""
    fields = [workloads.field_for("walk", (50000 + 1000 * i,), seed=970 + i) for i in range(6)]
    oas = [ref.compress(f, 1e-4, ref.EB_REL, 64, 256) for f in fields]
    bad = oas[3].copy()
    o = ref.sections(bad)["off_bits"]
    v = int.from_bytes(bad[o:o + 4].tobytes(), "little") + 64
    bad[o:o + 4] = np.frombuffer(v.to_bytes(4, "little"), np.uint8)
    arcs = [torch.from_numpy(a if i != 3 else bad).cuda() for i, a in enumerate(oas)]
    outs = [torch.empty(f.shape, dtype=torch.float32, device="cuda") for f in fields]
    with pytest.raises(gb.GbszError):
        ctx.decompress_batch(arcs, [a.size for a in oas], outs)
    import ctypes as C
    k = len(arcs)
    ap = (C.c_void_p * k)(*[a.data_ptr() for a in arcs])
    by = (C.c_size_t * k)(*[a.numel() for a in arcs])
    op = (C.c_void_p * k)(*[o_.data_ptr() for o_ in outs])
    caps = (C.c_uint64 * k)(*[o_.numel() for o_ in outs])
    sts = (C.c_int * k)()
    gb.load().gbsz_decompress_batch(ctx.h, k, ap, by, op, caps, sts, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert list(sts) == [0, 0, 0, gb.ERR_CORRUPT, 0, 0]
    for i in (0, 1, 2, 4, 5):
        assert np.array_equal(outs[i].cpu().numpy().view(np.uint32), ref.decompress(oas[i]).view(np.uint32)), i
