"""Device-memory accounting of a context (gbsz_memory_usage,
gbsz_release_scratch, gbsz_scratch_bytes), which the serving loop's budget
relies on: a fresh context holds one slot's fixed tables; a compress adds
exactly the field scratch gbsz_scratch_bytes states; a release returns to
the fixed tables, and the next call gives the oracle's bytes again."""
import numpy as np
import pytest
import torch

from oracle import ref
from paper_2007_09625_gb300 import serve, workloads

pytestmark = pytest.mark.gpu


def test_context_memory_matches_the_stated_scratch(gb):
    ctx = gb.Context(0)
    x = workloads.field_for("walk", (300007,), seed=61)
    field, slot = gb.scratch_bytes([x.size], 1e-4)
    assert ctx.memory_usage() == (slot, 1)
    xt = torch.from_numpy(x).cuda()
    arc, nb = ctx.compress(xt, 1e-4)
    torch.cuda.synchronize()
    assert ctx.memory_usage() == (slot + field, 1)
    want = ref.compress(x, 1e-4, ref.EB_REL, 512, gb.auto_chunk([x.size], 512))
    assert np.array_equal(arc[:nb].cpu().numpy(), want)
    y = ctx.decompress(arc, nb)
    torch.cuda.synchronize()
    dfield, _ = gb.scratch_bytes([x.size], 1e-4, for_decompress=True)
    used, _ = ctx.memory_usage()
    assert used <= slot + field + dfield
    ctx.release_scratch()
    assert ctx.memory_usage() == (slot, 1)
    arc2, nb2 = ctx.compress(xt, 1e-4)  # reallocates what it needs
    y2 = ctx.decompress(arc2, nb2)
    torch.cuda.synchronize()
    assert nb2 == nb and torch.equal(arc2[:nb2], arc[:nb])
    assert np.array_equal(y2.cpu().numpy().view(np.uint32), ref.decompress(want).view(np.uint32))
    assert torch.equal(y.view(torch.int32), y2.view(torch.int32))
    ctx.close()


def test_server_stays_within_its_budget(gb):
    """A budget that fits one big request at a time: the workers take turns,
    release their scratch to let each other run, and the counted memory
    never passes the budget; every result is the oracle's."""
    fields = [workloads.field_for("walk", (1_500_000 + 1000 * i,), seed=70 + i) for i in range(4)]
    field, slot = gb.scratch_bytes([fields[-1].size], 1e-3)
    budget = 3 * slot + int(1.5 * field)
    srv = serve.Server(workers=3, max_batch=4, mem_budget=budget).start()
    reqs = [srv.submit(serve.COMPRESS, torch.from_numpy(f).cuda(), eb=1e-3) for f in fields]
    for f, r in zip(fields, reqs):
        arc, nb = r.wait(120)
        want = ref.compress(f, 1e-3, ref.EB_REL, 512, gb.auto_chunk([f.size], 512))
        assert nb == want.size and np.array_equal(arc[:nb].cpu().numpy(), want)
    mem = srv.memory()
    srv.stop()
    assert mem["peak"] <= budget and mem["overruns"] == 0
