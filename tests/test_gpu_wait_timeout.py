"""Failure detection of the warp decoder's bounded wait, without a GPU fault:
the test hook withholds one chunk's look-back word, so the next chunk's wait
runs out after a second; the call must return TIMEOUT (not hang, not fault),
and the same context must then decode the archive exactly."""
import time

import numpy as np
import pytest
import torch

from oracle import ref
from paper_2007_09625_gb300 import workloads

pytestmark = pytest.mark.gpu


def test_withheld_lookback_word_times_out_and_context_recovers(gb):
    ctx = gb.Context(0)
    x = workloads.random_walk_1d(1 << 18, seed=1002)  # 64 chunks of 4096: the fused warp decoder
    t = torch.from_numpy(x).cuda()
    arc, nb = ctx.compress(t, 1e-4, gb.EB_REL, 512, 4096)
    torch.cuda.synchronize()
    y = torch.empty_like(t)
    for hold in (5, 0, 63):
        ctx.set_option(gb.OPT_TEST_HOLD_CHUNK, hold)
        t0 = time.perf_counter()
        st = ctx.decompress_status(arc, nb, y)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ctx.set_option(gb.OPT_TEST_HOLD_CHUNK, -1)
        if hold == 63:  # the last chunk: nobody waits for it
            assert st == gb.OK, gb.status_str(st)
        else:
            assert st == gb.ERR_TIMEOUT, gb.status_str(st)
            assert 0.9 < dt < 30.0, dt
        # the context still works, bit for bit
        st = ctx.decompress_status(arc, nb, y)
        torch.cuda.synchronize()
        assert st == gb.OK
        yo = ref.decompress(arc[:nb].cpu().numpy())
        assert np.array_equal(y.cpu().numpy().view(np.uint32), yo.view(np.uint32))
    with pytest.raises(gb.GbszError):
        ctx.set_option(gb.OPT_TEST_HOLD_CHUNK, -2)
    ctx.close()
