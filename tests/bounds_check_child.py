"""Run by test_gpu_bounds_check.py in a child process whose GBSZ_LIBRARY
names the bounds-checking build: every path of the library on fields of each
kind, compared with the oracle.  Prints one line per case, "ok <name>" or
"FAIL <name>: <why>", and exits 0."""
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import ref  # noqa: E402
from paper_2007_09625_gb300 import gbsz, workloads  # noqa: E402


def check_field(ctx, name, x, rel, R, C, lblock=0, order=1, decoders=(0, 1, 2, 3)):
    t = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    st = None
    try:
        arc, nb = ctx.compress(t, rel, gbsz.EB_REL, R, C, lblock=lblock, order=order)
        torch.cuda.synchronize()
    except gbsz.GbszError as e:
        return f"FAIL {name}: compress {e}"
    oa = ref.compress(x, rel, ref.EB_REL, R, C, lblock=lblock, order=order)
    if nb != oa.size or not np.array_equal(arc[:nb].cpu().numpy(), oa):
        return f"FAIL {name}: archive differs from the oracle's"
    yo = ref.decompress(oa)
    for dec in decoders:
        ctx.set_option(gbsz.OPT_DECODER, dec)
        y = torch.empty(x.shape, dtype=torch.float32, device="cuda")
        st = ctx.decompress_status(arc, nb, y)
        torch.cuda.synchronize()
        ctx.set_option(gbsz.OPT_DECODER, 0)
        if st != gbsz.OK:
            return f"FAIL {name}: decoder {dec} status {gbsz.status_str(st)}"
        if not np.array_equal(y.cpu().numpy().view(np.uint32), yo.view(np.uint32)):
            return f"FAIL {name}: decoder {dec} floats differ from the oracle's"
    return f"ok {name}"


def main():
    ctx = gbsz.Context(0)
    wf = workloads.field_for
    cases = [
        ("1d walk C64", wf("walk", (100003,), 1), 1e-4, 512, 64),
        ("1d walk C2048", wf("walk", (300007,), 2), 1e-4, 512, 2048),
        ("1d walk C8192", wf("walk", (100003,), 3), 1e-4, 512, 8192),
        ("1d long codes R32768", wf("walk", (50000,), 4), 1e-6, 32768, 1024),
        # from 2^23 points: code-0 bitmap and the separate outlier kernel
        ("1d walk bitmap C64", wf("walk", ((1 << 23) + 77,), 41), 1e-4, 512, 64),
        ("1d walk bitmap C16384", wf("walk", ((1 << 23) + 12345,), 42), 1e-4, 512, 16384),
        # anchored archives decoded straight to values by the thread decoder
        ("1d walk anchored C1024", wf("walk", ((1 << 23) + 4321,), 43), 1e-4, 512, 1024),
        ("1d walk anchored R2", wf("walk", ((1 << 20) + 9,), 44), 1e-4, 2, 2048),
        ("2d grf", wf("grf", (181, 1037), 5), 1e-3, 512, 4096),
        ("2d grf R32768", wf("grf", (300, 410), 6), 1e-5, 32768, 256),
        ("3d lognormal", wf("lognormal", (37, 41, 67), 7), 1e-4, 512, 256),
        ("3d sinus C4096", wf("sinus", (64, 64, 64), 8), 1e-4, 512, 4096),
        ("n=1", np.array([3.25], np.float32), 1e-3, 512, 64),
        ("tiny 3d", np.random.default_rng(0).normal(size=(2, 3, 5)).astype(np.float32), 1e-3, 2, 64),
        ("nonfinite", np.where(np.random.default_rng(3).random(5000) < 0.05, np.nan,
                               np.cumsum(np.random.default_rng(4).normal(size=5000))).astype(np.float32), 1e-3, 512, 64),
    ]
    for name, x, rel, R, C in cases:
        print(check_field(ctx, name, x, rel, R, C), flush=True)
    for name, x, lb, order in [("1d blocked", wf("walk", (70001,), 9), 1, 1), ("2d blocked", wf("sinus", (150, 170), 10), 1, 1),
                               ("3d order 2", wf("lognormal", (19, 23, 29), 11), 0, 2),
                               ("1d order 3", wf("walk", (40000,), 12), 0, 3)]:
        print(check_field(ctx, name, x, 1e-4, 512, 256, lblock=lb, order=order), flush=True)
    # 4D, folded to 3D
    x4 = wf("sinus", (3, 4, 19, 21), 13)
    print(check_field(ctx, "4d", x4, 1e-4, 512, 256), flush=True)
    # grouped batches, compress and decompress
    fields = [wf("walk", (30000 + 777 * i,), 20 + i) for i in range(5)] + [wf("grf", (90, 130), 30), wf("sinus", (17, 23, 29), 31)]
    ts = [torch.from_numpy(f).cuda() for f in fields]
    arcs, nbs, sts = ctx.compress_batch(ts, 1e-4, gbsz.EB_REL, 512, 256)
    torch.cuda.synchronize()
    ok = all(s == gbsz.OK for s in sts)
    oas = [ref.compress(f, 1e-4, ref.EB_REL, 512, 256) for f in fields]
    ok = ok and all(np.array_equal(a[:n].cpu().numpy(), o) for a, n, o in zip(arcs, nbs, oas))
    outs = [torch.empty_like(t) for t in ts]
    outs, dsts = ctx.decompress_batch(arcs, nbs, outs)
    torch.cuda.synchronize()
    ok = ok and all(s == gbsz.OK for s in dsts)
    ok = ok and all(np.array_equal(y.cpu().numpy().view(np.uint32), ref.decompress(o).view(np.uint32))
                    for y, o in zip(outs, oas))
    print(("ok" if ok else f"FAIL") + f" grouped batch {list(sts)} {list(dsts)}", flush=True)
    # corrupt archives are rejected as corrupt, never as an index failure
    x = wf("walk", (70001,), 40)
    bad_status = []
    for C in (256, 1024):  # and an anchored archive
        a = ref.compress(x, 1e-4, ref.EB_REL, 16, C)
        s = ref.sections(a)
        rng = np.random.default_rng(41 + C)
        for k in range(40):
            b = a.copy()
            b[int(rng.integers(s["off_anc"] if s["nanchor"] else s["off_str"], a.size))] ^= \
                np.uint8(1 << int(rng.integers(0, 8)))
            if k % 4 == 0:  # and an outlier index past the field
                o = s["off_out"] + 8 * (s["m"] - 1)
                b[o:o + 4] = np.frombuffer(np.uint32(0xFFFFFFF0).tobytes(), np.uint8)
            corrupt_status(ctx, b, x, k, C, bad_status)
    ctx.set_option(gbsz.OPT_DECODER, 0)
    print(("ok" if not bad_status else f"FAIL") + f" corrupt archives {bad_status[:5]}", flush=True)
    # the no-allocation codebook
    hist = np.bincount(ref.dualquant(x, ref.error_bound(x, 1e-4, ref.EB_REL), 512)["codes"], minlength=1024)
    ln, code, mx = gbsz.codebook_noalloc(torch.from_numpy(hist.astype(np.int32)).cuda())
    torch.cuda.synchronize()
    want, wmx = ref.huffman_lengths(hist.astype(np.uint32))
    print(("ok" if np.array_equal(ln.cpu().numpy(), want) and mx == wmx else "FAIL") + " no-alloc codebook", flush=True)
    ctx.close()


def corrupt_status(ctx, b, x, k, C, bad_status):
    """Every decoder reports the corrupt archive as OK or corrupt."""
    for dec in (0, 1, 2, 3):
        ctx.set_option(gbsz.OPT_DECODER, dec)
        st = ctx.decompress_status(torch.from_numpy(b).cuda(), b.size, torch.empty(x.shape, device="cuda"))
        torch.cuda.synchronize()
        if st not in (gbsz.OK, gbsz.ERR_CORRUPT):
            bad_status.append((C, k, dec, st))


if __name__ == "__main__":
    main()
