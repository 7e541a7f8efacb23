"""Benchmark: compress + decompress throughput of one FP32 field on GB300.

Workload (default): the 1D random walk of 2^28 values (1 GiB) with 1% spikes,
value-range-relative error bound 1e-4, radius 512 (1024 bins), Huffman
chunk by the library's rule (2048 symbols at 2^28).  One step = one compress and one decompress of the resident
field through the C ABI.  `value` = input bytes of all ranks / (max over
ranks of the timed K steps), in GB/s (1e9 bytes/s).

Under torchrun every rank compresses its own field (seed + rank): the
problems are independent, so there is no data-path collective (weak
scaling); only the timing is reduced (max over ranks).

--impl reference times the CPU oracle on the host cores instead, on a
bounded prefix of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compress+decompress GB/s (input FP32 bytes)"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--log2n", type=int, default=28, help="field size 2^k (default: the 2^28 workload)")
    ap.add_argument("--rel", type=float, default=1e-4)
    ap.add_argument("--radius", type=int, default=512)
    ap.add_argument("--chunk", type=int, default=0, help="0 = the library's rule (2048 at 2^28)")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--cpu-sample-log2", type=int, default=28,
                    help="CPU oracle sample: the first 2^k values of the workload (default: all of it)")
    ap.add_argument("--skip-batch", action="store_true",
                    help="skip the batched vs per-field measurement (16 x 1800x3600 fields)")
    ap.add_argument("--skip-micro", action="store_true",
                    help="skip the codebook-vs-bins and 32/64-bit codeword micro-benchmarks")
    ap.add_argument("--skip-serving", action="store_true", help="skip the serving-mix measurement")
    ap.add_argument("--skip-tune", action="store_true", help="skip the autotuner measurement")
    ap.add_argument("--oracle-configs", action="store_true",
                    help="also time the oracle (one thread and every host core) on the 64^3, 16 x 1800x3600 "
                         "and 512^3 workloads (about a minute of host time)")
    ap.add_argument("--skip-configs", action="store_true",
                    help="skip the other single-field workloads (64^3, 1800x3600, 512^3)")
    return ap.parse_args()


def batch_vs_per_field(ctx, gbsz, workloads, dev, steps=5):
    """16 fields of 1800x3600 (power-law -3 fields, four of them with masked
    constant regions) at rel eb 1e-4, and at 1e-3 beside it: one
    compress+decompress per field in a loop, versus one compress_batch +
    decompress_batch over all 16."""
    import torch
    fields = [torch.from_numpy(f).to(dev) for f in workloads.grf_2d_batch(16, seed=1003)]
    res = batch_at(ctx, gbsz, fields, 1e-4, dev, steps)
    res["rel_1e-3"] = batch_at(ctx, gbsz, fields, 1e-3, dev, steps)
    return res


def batch_at(ctx, gbsz, fields, rel, dev, steps):
    import torch
    n_all = sum(f.numel() for f in fields)
    params = [gbsz.make_params(gbsz.field_dims(f), rel) for f in fields]
    arcs = [torch.empty(gbsz.compress_bound(gbsz.field_dims(f), rel), dtype=torch.uint8, device=dev)
            for f in fields]
    outs = [torch.empty_like(f) for f in fields]
    # a stream of its own: batch calls on it are captured once as CUDA graphs
    # and replayed (the legacy default stream cannot be captured)
    stream = torch.cuda.Stream(dev)
    stream.wait_stream(torch.cuda.current_stream(dev))

    def per_field():
        for f, a, o in zip(fields, arcs, outs):
            _, nb = ctx.compress(f, rel, out=a, stream=stream)
            ctx.decompress(a, nb, out=o, stream=stream)

    def batched():
        _, nbs, _ = ctx.compress_batch(fields, None, outs=arcs, params=params, stream=stream)
        ctx.decompress_batch(arcs, nbs, outs, stream=stream)

    res = {}
    g0 = ctx.debug_copy(gbsz.DEBUG_GRAPHS, 4, np.uint64)
    for name, fn in (("per_field", per_field), ("batched", batched)):
        for _ in range(2):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        res[name] = 4.0 * n_all / (e0.elapsed_time(e1) / steps / 1e3) / 1e9
    # batched (graph-replayed) results are the single-field results
    single, nb1 = ctx.compress(fields[5], rel, stream=stream)
    _, nbs, _ = ctx.compress_batch(fields, None, outs=arcs, params=params, stream=stream)
    stream.synchronize()
    assert nbs[5] == nb1 and torch.equal(arcs[5][:nb1], single[:nb1])
    y5 = ctx.decompress(arcs[5], nbs[5], stream=stream)
    ctx.decompress_batch(arcs, nbs, outs, stream=stream)
    stream.synchronize()
    assert torch.equal(outs[5].view(torch.int32), y5.view(torch.int32))
    g1 = ctx.debug_copy(gbsz.DEBUG_GRAPHS, 4, np.uint64)
    return {"workload": f"16 x 1800x3600 FP32 power-law fields, rel eb {rel:g}, radius 512",
            "compression_ratio": 4.0 * n_all / float(sum(nbs)),
            "per_field_gbs": res["per_field"], "batched_gbs": res["batched"],
            "speedup": res["batched"] / res["per_field"], "steps": steps,
            "graph_replays": int(g1[1] - g0[1] + g1[3] - g0[3])}


def codebook_vs_bins(ctx, gbsz, dev, reps=5):
    """Codebook build time against the number of bins (2R = 128 .. 65536),
    the paper's codebook micro-benchmark (Sec. 3.2.2, its evaluation of the
    codebook stage): a white-noise field of 2^22 points with an absolute eb
    of 2.12 / R, so the residuals spread over most of the bins (residual
    standard deviation about R / 3)."""
    import torch
    g = torch.Generator(device=dev)
    g.manual_seed(1006)
    x = torch.randn(1 << 22, generator=g, device=dev, dtype=torch.float32)
    out = []
    for R in [64 << k for k in range(10)]:
        eb = 2.12 / R
        arc = torch.empty(gbsz.compress_bound([x.numel()], eb, gbsz.EB_ABS, R, 4096), dtype=torch.uint8, device=dev)
        ctx.compress(x, eb, gbsz.EB_ABS, R, 4096, out=arc)  # warm-up
        torch.cuda.synchronize(dev)
        ctx.profile_read()
        ctx.profile_enable(True)
        for _ in range(reps):
            ctx.compress(x, eb, gbsz.EB_ABS, R, 4096, out=arc)
        ms, calls, _ = ctx.profile_read()
        ctx.profile_enable(False)
        hist = ctx.debug_copy(gbsz.DEBUG_HIST, 2 * R, np.uint32)
        out.append({"bins": 2 * R, "used_bins": int((hist > 0).sum()),
                    "codebook_us": 1e3 * ms[2] / max(calls[2], 1)})
    return {"workload": "2^22 N(0,1) white noise, abs eb 2.12/R, chunk 4096", "points": out}


def encode_width(ctx, gbsz, x, eb, radius, chunk, dev, reps=5):
    """Encode (bit counts + offset scan + pack) with the adaptive 32-bit
    codeword entries against forced 64-bit entries (the paper's enc.32 /
    enc.64 comparison), on the benchmark's own field; the archives must be
    the same bytes."""
    import torch
    res = {}
    arcs = {}
    for name, width in (("enc32", 0), ("enc64", 64)):
        ctx.set_option(gbsz.OPT_CODEWORD_BITS, width)
        try:
            arc = torch.empty(gbsz.compress_bound([x.numel()], eb, gbsz.EB_REL, radius, chunk), dtype=torch.uint8,
                              device=dev)
            _, nb = ctx.compress(x, eb, gbsz.EB_REL, radius, chunk, out=arc)
            torch.cuda.synchronize(dev)
            ctx.profile_read()
            ctx.profile_enable(True)
            for _ in range(reps):
                _, nb = ctx.compress(x, eb, gbsz.EB_REL, radius, chunk, out=arc)
            ms, calls, _ = ctx.profile_read()
            ctx.profile_enable(False)
        finally:
            ctx.set_option(gbsz.OPT_CODEWORD_BITS, 0)
        enc_ms = sum(ms[3:6]) / reps
        res[name] = {"encode_ms": enc_ms, "encode_gbs": 4.0 * x.numel() / (enc_ms / 1e3) / 1e9,
                     "pack_ms": ms[5] / reps}
        arcs[name] = (arc, nb)
    (a32, n32), (a64, n64) = arcs["enc32"], arcs["enc64"]
    res["same_bytes"] = bool(n32 == n64 and torch.equal(a32[:n32], a64[:n64]))
    return res


def serving(gbsz, workloads, serve, dev, requests=256, rate=200.0, max_bytes=512 << 20, budget=64 << 30):
    """The serving mix as the workload states it: 256 seeded fields (rank
    1/2/3 uniform, sizes log-uniform 256 KiB - 512 MiB, generators of
    workloads 1-4, rel eb from {1e-2, 1e-3, 1e-4}), Poisson arrivals at 200
    req/s, half compress and half decompress (a decompress request takes the
    archive of its field compressed beforehand), a 64 GB device-memory budget
    over the workers' contexts.  p50 / p99 latency, throughput, mean batch and
    the counted memory at the offered rate, at 10x that rate and with every
    request submitted at once; every served result compared with the same
    request run alone (bit equality).  Fields are generated on the device."""
    import time
    import torch
    desc = workloads.serving_mix(count=requests, seed=1005, max_bytes=max_bytes)
    gens = {1: "sinus", 2: "walk", 3: "grf", 4: "lognormal"}
    fields = []
    for d in desc:
        kind = gens[d["gen"]]
        if d["rank"] == 1:
            kind = "walk"
        elif kind == "walk":
            kind = "sinus"
        fields.append(workloads.field_on_device(kind, d["shape"], 2000 + d["id"], dev).contiguous())
    alone = gbsz.Context(dev.index or 0)
    ref_arc, ref_out = [], []
    for f, d in zip(fields, desc):
        a, nb = alone.compress(f, d["rel"])
        ref_arc.append((a[:nb].clone(), nb))
        ref_out.append(alone.decompress(a, nb) if d["kind"] == "decompress" else None)
        del a
    torch.cuda.synchronize(dev)
    alone.close()
    field_bytes = sum(f.numel() * 4 for f in fields)
    arrivals = [d["arrival"] for d in desc]

    def run(scale):
        """scale: arrival times divided by it (None: all at once)"""
        srv = serve.Server(workers=2, max_batch=8, mem_budget=budget).start()
        outs = [torch.empty(ref_arc[i][1] + 64, dtype=torch.uint8, device=dev) if d["kind"] == "compress"
                else torch.empty_like(fields[i]) for i, d in enumerate(desc)]
        torch.cuda.synchronize(dev)
        reqs = []
        t0 = time.perf_counter()
        for i, d in enumerate(desc):
            if scale is not None:
                wait_s = arrivals[i] / scale - (time.perf_counter() - t0)
                if wait_s > 0:
                    time.sleep(wait_s)
            if d["kind"] == "compress":
                reqs.append(srv.submit(serve.COMPRESS, fields[i], eb=d["rel"], out=outs[i]))
            else:
                a, nb = ref_arc[i]
                reqs.append(srv.submit(serve.DECOMPRESS, a, nbytes=nb, out=outs[i]))
        equal = True
        for i, (d, r) in enumerate(zip(desc, reqs)):
            out = r.wait(600)
            if d["kind"] == "compress":
                arc, nb = out
                equal &= nb == ref_arc[i][1] and torch.equal(arc[:nb], ref_arc[i][0])
            else:
                equal &= torch.equal(out.view(torch.int32), ref_out[i].view(torch.int32))
        st = srv.stats()
        mem = srv.memory()
        srv.stop()
        del outs
        keep = ("requests", "p50_ms", "p99_ms", "throughput_gbs", "mean_batch", "span_s")
        res = {k: st[k] for k in keep}
        res.update({"peak_counted_gb": mem["peak"] / 1e9, "scratch_releases": mem["releases"],
                    "over_estimate": mem["overruns"], "bit_equal_to_alone": bool(equal)})
        return res

    offered = run(1.0)
    tenx = run(10.0)
    burst = run(None)
    return {"workload": f"{requests} fields of rank 1-3, 256 KiB-{max_bytes >> 20} MiB log-uniform "
                        f"({field_bytes / 1e9:.1f} GB in all), rel eb 1e-2/1e-3/1e-4, half compress, "
                        f"Poisson {rate:g} req/s, {budget >> 30} GiB budget, 2 workers, batches of up to 8",
            "offered": offered, "offered_x10": tenx, "all_at_once": burst,
            "note": "at 200 req/s a request's GPU work (about 0.2 ms for the mean 67 MiB field) is far "
                    "shorter than the mean gap between arrivals (5 ms), so requests rarely overlap; "
                    "the 10x and all-at-once runs show the batching"}


def other_configs(ctx, gbsz, workloads, dev, reps=5):
    """The other single-field workloads, compress and decompress of one
    resident field each, radius 512 unless stated, automatic chunk: 64^3
    sinusoids and one 1800x3600 power-law field at rel eb 1e-4; 64^3 at chunk
    4096 as the workload states it; the 512^3 lognormal density at rel eb
    1e-2, 1e-3, 1e-4 and 1e-5, each at radius 512 and 32768.  Per point:
    compress and decompress GB/s, compression ratio, max |x - x'| / eb."""
    import torch
    sin64 = lambda: workloads.sinusoids_3d(64, seed=1001)
    cases = [("64^3 sinusoids + noise (3D)", sin64, 1e-4, 512, 0),
             ("64^3 sinusoids + noise (3D), chunk 4096", sin64, 1e-4, 512, 4096),
             ("1800x3600 power-law field (2D)", lambda: workloads.grf_2d_batch(nfields=1, seed=1003, masked=(0,))[0],
              1e-4, 512, 0)]
    for R in (512, 32768):
        for rel in (1e-2, 1e-3, 1e-4, 1e-5):
            cases.append((f"512^3 lognormal density (3D), rel eb {rel:g}, radius {R}", "lognormal512", rel, R, 0))
    out = []
    stream = torch.cuda.Stream(dev)  # capturable: repeated calls replay as CUDA graphs
    cache = {}
    for name, make, rel, R, chunk in cases:
        if isinstance(make, str):
            if make not in cache:
                cache.clear()
                cache[make] = torch.from_numpy(workloads.lognormal_3d(512, seed=1004)).to(dev)
            x = cache[make]
        else:
            cache.clear()
            x = torch.from_numpy(make()).to(dev)
        dims = gbsz.field_dims(x)
        arc = torch.empty(gbsz.compress_bound(dims, rel, gbsz.EB_REL, R, chunk), dtype=torch.uint8, device=dev)
        y = torch.empty_like(x)
        torch.cuda.synchronize(dev)
        for _ in range(3):
            _, nb = ctx.compress(x, rel, gbsz.EB_REL, R, chunk, out=arc, stream=stream)
            ctx.decompress(arc, nb, out=y, stream=stream)
        stream.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        for _ in range(reps):
            ctx.compress(x, rel, gbsz.EB_REL, R, chunk, out=arc, stream=stream)
        ev[1].record(stream)
        for _ in range(reps):
            ctx.decompress(arc, nb, out=y, stream=stream)
        ev[2].record(stream)
        torch.cuda.synchronize(dev)
        cms, dms = ev[0].elapsed_time(ev[1]) / reps, ev[1].elapsed_time(ev[2]) / reps
        eb = float(np.frombuffer(arc[56:60].cpu().numpy().tobytes(), np.float32)[0])
        fin = torch.isfinite(x)
        err = float((x.double() - y.double()).abs()[fin].max()) / eb
        gb_ = x.numel() * 4 / 1e9
        out.append({"workload": name, "bytes": x.numel() * 4, "rel_eb": rel, "radius": R,
                    "chunk": chunk or gbsz.auto_chunk(dims, R), "ms_per_step": cms + dms,
                    "gbs": gb_ / ((cms + dms) / 1e3), "compress_gbs": gb_ / (cms / 1e3),
                    "decompress_gbs": gb_ / (dms / 1e3), "compression_ratio": x.numel() * 4 / nb,
                    "max_err_over_eb": err})
        del y, arc
    cache.clear()
    return out


def autotuned(gbsz, workloads, dev, reps=5):
    """The autotuner on three of the stated workloads (64^3 sinusoids, one
    1800x3600 power-law field, the 512^3 lognormal density; rel eb 1e-4,
    radius 512): compress + decompress GB/s with the built-in rules, then the
    tuner's choice (chunk, decoder, dual-quant tile extent) and the GB/s with
    it, in a context of its own."""
    import time
    import torch
    cases = [("64^3 sinusoids + noise (3D)", lambda: workloads.sinusoids_3d(64, seed=1001)),
             ("1800x3600 power-law field (2D)", lambda: workloads.grf_2d_batch(nfields=1, seed=1003, masked=(0,))[0]),
             ("512^3 lognormal density (3D)", lambda: workloads.lognormal_3d(512, seed=1004))]
    ctx = gbsz.Context(torch.device(dev).index or 0)
    stream = torch.cuda.Stream(dev)
    out = []

    def gbs(x, p):
        arc = torch.empty(gbsz.load().gbsz_compress_bound(gbsz.C.byref(p)), dtype=torch.uint8, device=dev)
        y = torch.empty_like(x)
        for _ in range(3):
            _, nb = ctx.compress_params(x, p, out=arc, stream=stream)
            ctx.decompress(arc, nb, out=y, stream=stream)
        stream.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(reps):
            _, nb = ctx.compress_params(x, p, out=arc, stream=stream)
            ctx.decompress(arc, nb, out=y, stream=stream)
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        return x.numel() * 4 / 1e9 / (ev[0].elapsed_time(ev[1]) / reps / 1e3)

    for name, make in cases:
        x = torch.from_numpy(make()).to(dev)
        rule = gbsz.make_params(gbsz.field_dims(x), 1e-4, gbsz.EB_REL, 512, 0)
        rule.chunk = gbsz.auto_chunk(gbsz.field_dims(x), 512)
        before = gbs(x, rule)
        t0 = time.perf_counter()
        p, _ = ctx.autotune(x, 1e-4, stream=stream)
        tune_s = time.perf_counter() - t0
        chunk, decoder, slab = ctx.tuned_knobs(p)
        after = gbs(x, p)
        out.append({"workload": name, "rule": {"chunk": rule.chunk, "gbs": before},
                    "tuned": {"chunk": chunk, "decoder": {0: "not measured", 1: "thread per chunk",
                                                          2: "warp per chunk"}[decoder],
                              "slab": slab or "rule", "gbs": after},
                    "tune_seconds": tune_s})
        del x
    ctx.close()
    return out


def oracle_configs(gbsz, workloads):
    """The oracle on the host cores, single-threaded and OpenMP, compress and
    decompress GB/s of input: 64^3 sinusoids (the rule's chunk and 4096),
    the 16 1800x3600 fields at rel 1e-3 and 1e-4 (all 16 per step), and the
    512^3 lognormal density at rel 1e-2..1e-5, radius 512 and 32768."""
    from oracle import ref
    sin64 = workloads.sinusoids_3d(64, seed=1001)
    grf = workloads.grf_2d_batch(16, seed=1003)
    logn = workloads.lognormal_3d(512, seed=1004)
    cases = [("64^3 sinusoids, rel 1e-4, chunk 64", [sin64], 1e-4, 512, 64),
             ("64^3 sinusoids, rel 1e-4, chunk 4096", [sin64], 1e-4, 512, 4096)]
    for rel in (1e-3, 1e-4):
        cases.append((f"16 x 1800x3600, rel {rel:g}", grf, rel, 512, gbsz.auto_chunk([3600, 1800], 512)))
    for R in (512, 32768):
        for rel in (1e-2, 1e-3, 1e-4, 1e-5):
            cases.append((f"512^3 lognormal, rel {rel:g}, radius {R}", [logn], rel, R,
                          gbsz.auto_chunk([512, 512, 512], R)))
    out = []
    for name, fields, rel, R, chunk in cases:
        nbytes = 4 * sum(f.size for f in fields)
        row = {"workload": name, "cores_omp": ref.threads(omp=True)}
        for omp in (False, True):
            tc = td = 0.0
            size = 0
            for f in fields:
                t0 = time.perf_counter()
                arc = ref.compress(f, rel, ref.EB_REL, R, chunk, omp=omp)
                t1 = time.perf_counter()
                ref.decompress(arc, omp=omp)
                t2 = time.perf_counter()
                tc, td, size = tc + t1 - t0, td + t2 - t1, size + arc.size
            row["omp" if omp else "single"] = {"compress_gbs": nbytes / tc / 1e9, "decompress_gbs": nbytes / td / 1e9}
            row["compression_ratio"] = nbytes / size
        out.append(row)
    return out


def workload_chunk(n):
    """The Huffman chunk the library's rule picks for n points (chunk = 0):
    the smallest power of two in 64..4096 whose chunks fit in one wave of
    1024 decoding threads per SM on a 152-SM GB300.  Both arms of the
    benchmark use it, so they run the same configuration."""
    c = 64
    while c < 4096 and c * 152 * 1024 < n:
        c *= 2
    return c


def workload_config(a, n, chunk):
    return {"workload": f"1D random walk 2^{a.log2n} FP32 (1% spikes), rel eb {a.rel:g}, radius {a.radius}, "
                        f"chunk {chunk}", "n": n, "eb_mode": "rel", "eb": a.rel, "radius": a.radius,
            "chunk": chunk, "l2": "inputs larger than L2 (1 GiB field vs 129 MB L2)" if n * 4 > (256 << 20)
            else "input smaller than L2; no flush", "parallelism": "replicas (one field per rank)"}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of each
# stage's kernels (pack: pack + outliers) on the full 2^28-point walk, from one
# ncu capture, with a digest of the sources the kernels were built from; a
# number is reported only while those sources are unchanged.
DRAM_TRAFFIC = {
    "error_bound": (1079894528, ('k_quant.cu', 'common.cuh'), "46464c23b2bc0113"),
    "dualquant_hist": (1749994325, ('k_quant.cu', 'common.cuh'), "46464c23b2bc0113"),
    "encode_count": (572855893, ('k_encode.cu', 'common.cuh', 'scan.cuh'), "eafb965bd833f037"),
    "encode_pack": (929418922, ('k_encode.cu', 'common.cuh', 'scan.cuh'), "eafb965bd833f037"),
    "decode": (1248666709, ('k_decode.cu', 'common.cuh', 'scan.cuh'), "362706e8664691c7"),
}
TRAFFIC_CONFIG = (28, 1e-4, 512, 2048)  # log2 n, rel eb, radius, chunk of the capture


def measured_traffic(stage, config):
    """DRAM bytes per launch from the table above, or None if the workload
    differs or the kernel's sources changed since the capture."""
    import hashlib
    ent = DRAM_TRAFFIC.get(stage)
    if ent is None or tuple(config) != TRAFFIC_CONFIG:
        return None
    nbytes, files, digest = ent
    h = hashlib.sha256()
    base = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2007_09625_gb300", "csrc")
    for f in files:
        with open(os.path.join(base, f), "rb") as fh:
            h.update(fh.read())
    return nbytes if h.hexdigest()[:16] == digest else None


def read_peaks():
    try:
        with open(PEAKS) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region (clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(rank):
    """Every rank compresses its own field: workload seed 1002 + rank."""
    return 1002 + rank


def reduce_max(value, device):
    """Max over ranks of a timing (the only collective of the benchmark)."""
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_time(x, a, chunk, omp=False):
    from oracle import ref
    t0 = time.perf_counter()
    arc = ref.compress(x, a.rel, ref.EB_REL, a.radius, chunk, omp=omp)
    t1 = time.perf_counter()
    ref.decompress(arc, omp=omp)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1, arc.size


def cpu_sample_text(ns, n_full, what):
    whole = "the whole workload" if ns == n_full else "the first"
    return f"{whole} ({'2^%d' % (ns.bit_length() - 1)} values), {what}"


def run_reference(a):
    """The oracle's OpenMP build on the host cores, compress + decompress of
    the workload (or a prefix of it) per step."""
    from oracle import ref
    from paper_2007_09625_gb300 import workloads
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    n_full = 1 << a.log2n
    ns = min(n_full, 1 << a.cpu_sample_log2)
    x = workloads.random_walk_1d(n_full, seed=1002)[:ns].copy()
    chunk = a.chunk or workload_chunk(n_full)
    for _ in range(a.warmup):
        cpu_oracle_time(x, a, chunk, omp=True)
    ts = []
    for _ in range(a.steps):
        tc, td, nb = cpu_oracle_time(x, a, chunk, omp=True)
        ts.append(tc + td)
    t = float(np.mean(ts))
    gbs = 4 * ns / t / 1e9
    line = {"metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "reference",
            "config": workload_config(a, n_full, chunk),
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": ref.threads(omp=True), "kind": "oracle",
                             "sample": cpu_sample_text(ns, n_full, "compress+decompress per step, "
                                                                  "OpenMP build of the oracle")},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    import torch

    from paper_2007_09625_gb300 import gbsz, workloads

    ws, rank, local = dist_env()
    dist = ws > 1
    if dist:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = 1 << a.log2n
    x_host = workloads.random_walk_1d(n, seed=rank_seed(rank))
    x = torch.from_numpy(x_host).to(dev)
    ctx = gbsz.Context(local)
    chunk = a.chunk or gbsz.auto_chunk([n], a.radius)
    assert a.chunk or chunk == workload_chunk(n), "chunk rule differs between the arms"
    bound = gbsz.compress_bound([n], a.rel, gbsz.EB_REL, a.radius, chunk)
    arc = torch.empty(bound, dtype=torch.uint8, device=dev)
    y = torch.empty_like(x)
    # a stream of its own: repeated calls on the same buffers are captured as
    # CUDA graphs by the library (after two eager calls) and replayed, stage
    # timing events included
    stream = torch.cuda.Stream(dev)

    def step():
        _, nb = ctx.compress(x, a.rel, gbsz.EB_REL, a.radius, chunk, out=arc, stream=stream)
        ctx.decompress(arc, nb, out=y, stream=stream)
        return nb

    torch.cuda.synchronize(dev)  # inputs and buffers made on the default stream are ready
    for _ in range(max(a.warmup, 0)):
        nb = step()
    torch.cuda.synchronize(dev)
    # correctness of the timed configuration: error bound on every element
    err = (x.double() - y.double()).abs()
    hdr = arc[:128].cpu().numpy()
    ebf = float(np.frombuffer(hdr[56:60].tobytes(), np.float32)[0])  # header: eb
    maxlen = int(np.frombuffer(hdr[104:108].tobytes(), np.uint32)[0])  # header: longest code
    fin = torch.isfinite(x)
    max_err = float(err[fin].max())
    assert max_err <= ebf, "error bound violated"
    xf = x[fin].double()
    vrange = float(xf.max() - xf.min())
    mse = float((err[fin] ** 2).mean())
    psnr = 20 * np.log10(vrange) - 10 * np.log10(mse) if mse > 0 and vrange > 0 else float("inf")
    del err, xf

    ctx.profile_read()  # reset counters
    ctx.profile_enable(True)
    sampler = ClockSampler(local)
    if dist:
        tdist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        nb = step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    if dist:
        tdist.barrier()
    ms_total = e0.elapsed_time(e1)
    stage_ms, stage_calls, launches = ctx.profile_read()
    ctx.profile_enable(False)
    if dist:
        ms_total = reduce_max(ms_total, dev)
    ms_step = ms_total / a.steps
    value = 4.0 * n * ws / (ms_step / 1e3) / 1e9

    # compress-only and decompress-only times from the stage events
    comp_ms = sum(stage_ms[0:6]) / a.steps
    dec_ms = sum(stage_ms[6:10]) / a.steps
    cr = 4.0 * n / nb

    # roofline of the dominant stage (algorithmic bytes per launch, below)
    peaks, peak_kind = read_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    m_out = int(np.frombuffer(arc[80:88].cpu().numpy().tobytes(), np.uint64)[0])
    w_words = int(np.frombuffer(arc[96:104].cpu().numpy().tobytes(), np.uint64)[0])
    f = m_out / n
    nc = (n + chunk - 1) // chunk
    # From 2^23 points the library's 1D order-1 path keeps a code-0 bitmap:
    # the count kernel writes it (n/8 bytes) and the pack stage is pack plus
    # k_encode_outliers, which reads it back with the residuals.
    zb = n >= (1 << 23)
    bm = n / 8.0 if zb else 0.0
    # Archives of 1D fields in chunks of >= 1024 symbols carry chunk anchors;
    # with codes of at most 15 bits and more chunks than the warp decoder
    # takes (32 per SM), the library's thread decoder writes the values
    # itself (each chunk from its anchor): decode reads the stream, the chunk
    # table, offsets, anchors, outlier starts and records and writes the
    # field, and no separate reconstruction runs.
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fused = chunk >= 1024 and maxlen <= 15 and nc > 32 * sms
    alg = {  # algorithmic bytes per launch of each stage (one kernel, or pack + outliers)
        0: 4.0 * n,                                               # minmax: read the field
        1: 6.0 * n + 8.0 * m_out,                                 # dual-quant: field in, codes out, residuals
        3: 2.0 * n + n / 32.0 + 4.0 * nc + bm,                    # count: codes in; lane bits, chunk bits (bitmap) out
        5: 2.0 * n + n / 32.0 + 16.0 * m_out + 4.0 * w_words + bm,  # pack: codes, lane bits, residuals (bitmap) in; stream, records out
        # decode: stream, bits, offsets in; codes out -- or, fused, the
        # anchors, outlier starts and records in and the values out
        8: (4.0 * w_words + 20.0 * nc + 8.0 * m_out + 4.0 * n) if fused else (4.0 * w_words + 12.0 * nc + 2.0 * n),
    }
    dom = max(alg, key=lambda s: stage_ms[s])
    dom_ms = stage_ms[dom] / max(stage_calls[dom], 1)
    achieved = alg[dom] / (dom_ms / 1e3) / 1e9
    stage_names = gbsz.STAGES
    roofline = {"bound": "hbm", "kernel": stage_names[dom], "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm, "peak_kind": f"{peak_kind} (MEASURED_PEAKS hbm_gbs)",
                "traffic": measured_traffic(stage_names[dom], (a.log2n, a.rel, a.radius, chunk)),
                "alg_bytes_per_launch": alg[dom]}
    # the whole compress+decompress step: 12 + 8f + 4/CR (compress, relative
    # eb) plus, for decompress, 8 + 8f + 4/CR bytes per point with the codes
    # written and read back, or 4 + 8f + 4/CR when the decoder writes the
    # values itself
    cbytes = n * (12.0 + 8.0 * f + 4.0 / cr)
    dbytes = n * ((4.0 if fused else 8.0) + 8.0 * f + 4.0 / cr)
    step_bytes = cbytes + dbytes
    pipe_gbs = step_bytes / (ms_step / 1e3) / 1e9
    pipe = {"alg_bytes_per_step": step_bytes, "achieved_gbs": pipe_gbs, "peak": hbm, "frac": pipe_gbs / hbm,
            "decompress_fused": fused}
    if comp_ms and dec_ms:
        pipe["compress_frac"] = cbytes / (comp_ms / 1e3) / 1e9 / hbm
        pipe["decompress_frac"] = dbytes / (dec_ms / 1e3) / 1e9 / hbm
        # against the two-kernel path's bytes (8 + 8f + 4/CR), for comparison
        # with a decompress that writes the codes
        pipe["decompress_frac_two_kernel_bytes"] = n * (8.0 + 8.0 * f + 4.0 / cr) / (dec_ms / 1e3) / 1e9 / hbm
    # every single-kernel stage against the same peak
    per_kernel = {}
    for st_i, by in alg.items():
        ms1 = stage_ms[st_i] / max(stage_calls[st_i], 1)
        gbs = by / (ms1 / 1e3) / 1e9 if ms1 > 0 else 0.0
        per_kernel[stage_names[st_i]] = {"ms": ms1, "alg_gbs": gbs, "frac": gbs / hbm,
                                         "traffic": measured_traffic(stage_names[st_i],
                                                                     (a.log2n, a.rel, a.radius, chunk))}

    e2e = None
    if not a.skip_e2e:
        # Through the host-buffer entry points, every step: upload the field,
        # compress, download the archive (gbsz_compress_host), then upload the
        # archive, decompress and download the field
        # (gbsz_decompress_host_async).  Step k's field download runs while
        # step k+1's field uploads (two streams, archives double-buffered);
        # each step waits for the previous step's result before it starts
        # its own decompress.  All copies are from / to pinned host memory.
        hx = torch.from_numpy(x_host).pin_memory()
        harcs = [torch.empty(bound, dtype=torch.uint8).pin_memory() for _ in range(2)]
        hy = torch.empty_like(hx).pin_memory()
        sa, sb = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

        def pipelined(k_steps):
            hnb = 0
            for k in range(k_steps):
                _, hnb = ctx.compress_host(hx, a.rel, gbsz.EB_REL, a.radius, chunk, out=harcs[k % 2], stream=sa)
                ctx.async_wait()
                ctx.decompress_host_async(harcs[k % 2], hnb, hy, stream=sb)
            ctx.async_wait()
            return hnb

        def sequential(k_steps):
            hnb = 0
            for _ in range(k_steps):
                _, hnb = ctx.compress_host(hx, a.rel, gbsz.EB_REL, a.radius, chunk, out=harcs[0], stream=sa)
                ctx.decompress_host(harcs[0], hnb, hy, stream=sa)
            return hnb

        ke = max(1, min(a.steps, 8))
        times = {}
        for name, fn in (("pipelined", pipelined), ("sequential", sequential)):
            fn(2)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            hnb = fn(ke)
            torch.cuda.synchronize(dev)
            times[name] = (time.perf_counter() - t0) / ke
            assert torch.equal(hy.view(torch.int32), y.cpu().view(torch.int32))
        te = times["pipelined"]
        if dist:
            te = reduce_max(te, dev)
        e2e = {"value": 4.0 * n * ws / te / 1e9, "unit": "GB/s", "h2d_bytes_per_step": 4 * n + hnb,
               "d2h_bytes_per_step": hnb + 4 * n, "ms_per_step": te * 1e3, "steps": ke,
               "mode": "pipelined: step k's field download overlaps step k+1's upload",
               "sequential_gbs": 4.0 * n / times["sequential"] / 1e9}

    batch = None
    if not a.skip_batch:
        batch = batch_vs_per_field(ctx, gbsz, workloads, dev)

    micro = None
    if rank == 0 and not a.skip_micro:
        micro = {"codebook_vs_bins": codebook_vs_bins(ctx, gbsz, dev),
                 "codeword_width": encode_width(ctx, gbsz, x, a.rel, a.radius, chunk, dev)}

    configs_res = None
    if rank == 0 and not a.skip_configs:
        configs_res = other_configs(ctx, gbsz, workloads, dev)

    oracle_res = None
    if rank == 0 and a.oracle_configs:
        oracle_res = oracle_configs(gbsz, workloads)

    tune_res = None
    if rank == 0 and not a.skip_tune:
        tune_res = autotuned(gbsz, workloads, dev)

    serving_res = None
    if rank == 0 and not a.skip_serving:
        from paper_2007_09625_gb300 import serve
        serving_res = serving(gbsz, workloads, serve, dev)

    cpu = None
    if rank == 0 and not a.skip_cpu_baseline:
        from oracle import ref
        ns = min(n, 1 << a.cpu_sample_log2)
        xs = x_host[:ns]
        # the oracle's OpenMP build on every host core is the baseline; its
        # single-threaded build beside it
        tco, tdo, _ = cpu_oracle_time(xs, a, chunk, omp=True)
        tc, td, _ = cpu_oracle_time(xs, a, chunk)
        cpu = {"value": 4 * ns / (tco + tdo) / 1e9, "unit": "GB/s", "cores": ref.threads(omp=True),
               "kind": "oracle", "sample": cpu_sample_text(ns, n, "one compress+decompress, OpenMP build"),
               "compress_gbs": 4 * ns / tco / 1e9, "decompress_gbs": 4 * ns / tdo / 1e9,
               "single_thread": {"value": 4 * ns / (tc + td) / 1e9, "cores": 1,
                                 "compress_gbs": 4 * ns / tc / 1e9, "decompress_gbs": 4 * ns / td / 1e9}}
        cpu["omp_speedup"] = cpu["value"] / cpu["single_thread"]["value"]

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(a, n, chunk),
                "compress_gbs": 4.0 * n / (comp_ms / 1e3) / 1e9 if comp_ms else None,
                "decompress_gbs": 4.0 * n / (dec_ms / 1e3) / 1e9 if dec_ms else None,
                "compression_ratio": cr, "outlier_frac": f, "max_code_len": maxlen,
                "psnr_db": psnr, "max_err_over_eb": max_err / ebf,
                "pipeline_roofline": pipe,
                "stage_ms_per_step": {nm: stage_ms[i] / a.steps for i, nm in enumerate(stage_names)},
                "roofline": roofline, "kernels": per_kernel, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "batch_vs_per_field": batch, "micro": micro, "serving": serving_res,
                "other_single_field": configs_res, "autotune": tune_res, "oracle_configs": oracle_res,
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if dist:
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
