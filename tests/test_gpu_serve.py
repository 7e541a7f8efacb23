"""The serving loop on the GPU: a stream of mixed compress / decompress
requests arriving while others run gives, for every request, exactly the
bytes (archives) and floats (reconstructions) that the oracle gives for the
same input, and that the same request gives alone.  Integer / bit-exact
results, so the tolerance is equality."""
import time

import numpy as np
import pytest
import torch

from oracle import ref
from paper_2007_09625_gb300 import serve, workloads

pytestmark = pytest.mark.gpu


def test_mixed_stream_matches_alone(gb):
    rng = np.random.default_rng(77)
    kinds = ["walk", "sinus", "grf", "lognormal"]
    fields = []
    for i in range(24):
        rank = int(rng.integers(1, 4))
        nbytes = float(np.exp(rng.uniform(np.log(64 << 10), np.log(4 << 20))))
        n = max(64, int(nbytes // 4))
        if rank == 1:
            shape = (n,)
        elif rank == 2:
            a = int(np.sqrt(n))
            shape = (max(2, n // a), a)
        else:
            a = int(round(n ** (1 / 3)))
            shape = (max(2, n // (a * a)), a, a)
        kind = kinds[i % 4] if rank > 1 or kinds[i % 4] == "walk" else "walk"
        fields.append(workloads.field_for(kind, shape, seed=500 + i))
    rels = [1e-2, 1e-3, 1e-4]
    alone = gb.Context(0)
    ref_arcs, ref_out = [], []
    for i, f in enumerate(fields):
        a, nb = alone.compress(torch.from_numpy(f).cuda(), rels[i % 3])
        ref_arcs.append((a[:nb].clone(), nb))
        ref_out.append(alone.decompress(a, nb).cpu().numpy())
        # the oracle's archive and reconstruction for the same request
        chunk = gb.auto_chunk(list(f.shape)[::-1], 512)
        oa = ref.compress(f, rels[i % 3], ref.EB_REL, radius=512, chunk=chunk, omp=True)
        assert nb == oa.size and np.array_equal(a[:nb].cpu().numpy(), oa), i
        yo = ref.decompress(oa, omp=True)
        assert np.array_equal(ref_out[-1].view(np.uint32), yo.view(np.uint32)), i
    torch.cuda.synchronize()

    srv = serve.Server(workers=2, max_batch=4, mem_budget=2 << 30).start()
    reqs = []
    for i, f in enumerate(fields):
        x = torch.from_numpy(f).cuda()
        if i % 2 == 0:
            reqs.append(("c", i, srv.submit(serve.COMPRESS, x, eb=rels[i % 3])))
        else:
            a, nb = ref_arcs[i]
            reqs.append(("d", i, srv.submit(serve.DECOMPRESS, a, nbytes=nb)))
        time.sleep(float(rng.exponential(1 / 200.0)))
    for kind, i, r in reqs:
        out = r.wait(120)
        assert r.status == gb.OK
        if kind == "c":
            arc, nb = out
            assert nb == ref_arcs[i][1] and torch.equal(arc[:nb], ref_arcs[i][0]), i
        else:
            assert np.array_equal(out.cpu().numpy().view(np.uint32), ref_out[i].view(np.uint32)), i
    st = srv.stats()
    srv.stop()
    alone.close()
    assert st["requests"] == len(fields) and st["p99_ms"] >= st["p50_ms"]


def test_server_reports_per_request_errors_and_budget(gb):
    x = torch.from_numpy(workloads.field_for("walk", (300001,), seed=5)).cuda()
    alone = gb.Context(0)
    a, nb = alone.compress(x, 1e-4)
    y_alone = alone.decompress(a, nb)
    torch.cuda.synchronize()
    bad = a[:nb].clone()
    o = ref.sections(bad.cpu().numpy())["off_bits"]
    b0 = int(bad[o:o + 4].cpu().numpy().view(np.uint32)[0]) + 64  # chunk 0 claims two more words
    bad[o:o + 4] = torch.from_numpy(np.array([b0], np.uint32).view(np.uint8)).cuda()
    torch.cuda.synchronize()
    srv = serve.Server(workers=2, max_batch=2, mem_budget=64 << 20).start()
    good = srv.submit(serve.DECOMPRESS, a, nbytes=nb)
    broken = srv.submit(serve.DECOMPRESS, bad, nbytes=nb)
    comp = srv.submit(serve.COMPRESS, x, eb=1e-4)
    too_big = srv.submit(serve.COMPRESS, torch.zeros(8 << 20, device="cuda"), eb=1e-4)  # 12 B/point > 64 MiB
    assert torch.equal(good.wait(60).view(torch.int32), y_alone.view(torch.int32))
    with pytest.raises(gb.GbszError) as e:
        broken.wait(60)
    assert e.value.status == gb.ERR_CORRUPT
    arc, n2 = comp.wait(60)
    assert n2 == nb and torch.equal(arc[:n2], a[:nb])
    assert too_big.status == "rejected"
    with pytest.raises(MemoryError):
        too_big.wait(1)
    st = srv.stats()
    srv.stop()
    alone.close()
    assert st["requests"] == 2  # completed without error
