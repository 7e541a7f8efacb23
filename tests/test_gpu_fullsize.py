"""Full-size workloads on the GPU, archive and reconstruction compared with
the oracle byte for byte, in the launch configuration the benchmark uses
(automatic chunk, device-resident buffers, one context reused).

Sizes: 64^3 sinusoids; 2^28 random walk with 1% spikes (the benchmark
workload), also in the per-block Lorenzo mode; one 1800x3600 power-law field
at rel 1e-3 and 1e-4; 512^3 lognormal at rel 1e-2, 1e-3, 1e-4 and 1e-5, each
at radius 512 and 32768, and with the order-2 predictor; a field of the paper's 4D QMCPACK shape 288x115x69x69.  The oracle runs multi-threaded where
its loops allow; these tests take a few minutes.
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


def roundtrip_vs_oracle(gb, ctx, x, rel, R, order=1, lblock=0):
    n = x.size
    chunk = gb.auto_chunk(list(x.shape)[::-1], R)
    xt = torch.from_numpy(x).cuda()
    arc, nb = ctx.compress(xt, rel, gb.EB_REL, R, chunk, order=order, lblock=lblock)
    y = ctx.decompress(arc, nb)
    torch.cuda.synchronize()
    oa = ref.compress(x, rel, ref.EB_REL, radius=R, chunk=chunk, omp=True, order=order, lblock=lblock)
    ga = arc[:nb].cpu().numpy()
    if not (nb == oa.size and np.array_equal(ga, oa)):
        gs, os_ = ref.sections(ga), ref.sections(oa)
        for k in ("m", "e", "words", "maxlen"):
            assert gs[k] == os_[k], (k, gs[k], os_[k])
        for k in ("len", "bits", "out_idx", "out_delta", "exc_idx", "exc_raw", "stream"):
            if not np.array_equal(gs[k], os_[k]):
                bad = np.flatnonzero(gs[k] != os_[k]) if gs[k].shape == os_[k].shape else None
                raise AssertionError(f"section {k} differs; first {None if bad is None else bad[:8]}")
        raise AssertionError("archive bytes differ")
    yo = ref.decompress(oa, omp=True)
    yg = y.cpu().numpy()
    assert np.array_equal(yg.view(np.uint32), yo.view(np.uint32)), "reconstruction differs"
    eb = np.frombuffer(oa[56:60].tobytes(), np.float32)[0]
    fin = np.isfinite(x)
    assert np.abs(x[fin].astype(np.float64) - yg[fin]).max() <= eb
    return n * 4 / nb


def test_sinusoids_64cubed(gb, ctx):
    x = workloads.sinusoids_3d(64, seed=1001)
    roundtrip_vs_oracle(gb, ctx, x, 1e-4, 512)


def test_random_walk_2p28(gb, ctx):
    x = workloads.random_walk_1d(1 << 28, seed=1002)
    cr = roundtrip_vs_oracle(gb, ctx, x, 1e-4, 512)
    assert cr > 3


@pytest.mark.parametrize("rel", [1e-3, 1e-4])
def test_grf_1800x3600(gb, ctx, rel):
    x = workloads.grf_2d_batch(nfields=1, seed=1003, masked=(0,))[0]
    roundtrip_vs_oracle(gb, ctx, x, rel, 512)


@pytest.fixture(scope="module")
def lognormal512():
    return workloads.lognormal_3d(512, seed=1004)


# the 512^3 error-bound sweep: relative eb 1e-2 .. 1e-5 at 1024 and 65536 bins
@pytest.mark.parametrize("R", [512, 32768])
@pytest.mark.parametrize("rel", [1e-2, 1e-3, 1e-4, 1e-5])
def test_lognormal_512cubed(gb, ctx, lognormal512, rel, R):
    roundtrip_vs_oracle(gb, ctx, lognormal512, rel, R)


def test_random_walk_2p28_per_block(gb, ctx):
    x = workloads.random_walk_1d(1 << 28, seed=1002)
    roundtrip_vs_oracle(gb, ctx, x, 1e-4, 512, lblock=1)


def test_lognormal_512cubed_order2(gb, ctx, lognormal512):
    roundtrip_vs_oracle(gb, ctx, lognormal512, 1e-4, 512, order=2)


def test_qmcpack_shape_4d(gb, ctx):
    """288x115x69x69 (the paper's QMCPACK extents): a smooth separable field
    plus noise, predicted as 3D over the folded two slowest axes."""
    rng = np.random.default_rng(1007)
    a = np.arange(288, dtype=np.float32)[:, None, None, None]
    b = np.arange(115, dtype=np.float32)[None, :, None, None]
    c = np.arange(69, dtype=np.float32)[None, None, :, None]
    d = np.arange(69, dtype=np.float32)[None, None, None, :]
    x = np.sin(a / 7) + np.cos(b / 5) + np.sin(c / 3) * np.cos(d / 4)
    x = (x + rng.normal(0, 1e-3, x.shape).astype(np.float32)).astype(np.float32)
    roundtrip_vs_oracle(gb, ctx, x, 1e-4, 512)
