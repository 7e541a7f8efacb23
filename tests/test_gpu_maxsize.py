"""A field beyond 2^31 points (8.6 GB), the range where 32-bit signed index
arithmetic would break: checked by properties that hold at any size, since
the oracle cannot run it in seconds -- every value within the error bound,
the outlier count equal to the number of code-0 symbols (checked by the
library), two compressions byte-identical, and one decompression per
archive.  The field is a float32 random walk with spikes, made on the GPU."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

N = (1 << 31) + (1 << 20) + 7


def test_field_beyond_2p31_points(gb):
    free, _ = torch.cuda.mem_get_info()
    if free < (60 << 30):
        pytest.skip("needs about 60 GB of free device memory")
    g = torch.Generator(device="cuda")
    g.manual_seed(1008)
    x = torch.randn(N, generator=g, device="cuda", dtype=torch.float32).mul_(1e-2).cumsum_(0)
    spikes = torch.randint(0, N, (N // 100,), generator=g, device="cuda")
    x[spikes] = torch.rand(spikes.numel(), generator=g, device="cuda") * 900.0 - 450.0
    ctx = gb.Context(0)
    cap = 8 << 30
    a1 = torch.empty(cap, dtype=torch.uint8, device="cuda")
    _, nb1 = ctx.compress(x, 1e-4, gb.EB_REL, 512, 0, out=a1)
    a2 = torch.empty(nb1, dtype=torch.uint8, device="cuda")
    _, nb2 = ctx.compress(x, 1e-4, gb.EB_REL, 512, 0, out=a2)
    assert nb2 == nb1 and torch.equal(a1[:nb1], a2)
    del a2
    p, n = gb.archive_info(a1[:128].cpu().numpy(), nb1)
    assert n == N and p.dims[0] == N
    y = ctx.decompress(a1, nb1)
    torch.cuda.synchronize()
    eb = float(np.frombuffer(a1[56:60].cpu().numpy().tobytes(), np.float32)[0])
    step = 1 << 28
    worst = 0.0
    for i in range(0, N, step):
        d = (x[i:i + step].double() - y[i:i + step].double()).abs().max().item()
        worst = max(worst, d)
    assert worst <= eb, (worst, eb)
    ctx.close()
