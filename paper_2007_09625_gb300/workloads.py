"""Seeded synthetic FP32 fields shaped like the paper's evaluation data.

The paper evaluates on SDRBench fields (HACC 1D, CESM-ATM 2D 1800x3600,
Hurricane 3D 100x500x500, Nyx 3D 512^3, QMCPACK 4D; Table "datasets" of
Sec. 4.1), which are not available here.  These generators stand in for
them with the same shapes and comparable statistics.  They contain none of
the compressor's arithmetic and are shared by the tests, the smoke check and
the benchmark.  Seeds are 1000 + workload id; every array is C-ordered
(last axis fastest) float32.
"""
import numpy as np


def _fft():
    try:
        import scipy.fft as f
        return f, {"workers": -1}
    except Exception:  # pragma: no cover - scipy is present on both machines
        return np.fft, {}


def sinusoids_3d(n=64, seed=1001, n_waves=8, noise_rel=1e-3):
    """Workload 1: n^3 sum of 8 random-phase sinusoids plus Gaussian noise of
    sigma = noise_rel * value range."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
    f = np.zeros((n, n, n), np.float64)
    for _ in range(n_waves):
        k = rng.integers(1, 9, 3)
        a = rng.uniform(0.5, 1.0)
        ph = rng.uniform(0, 2 * np.pi)
        f += a * np.sin(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z) / n + ph)
    rngv = f.max() - f.min()
    f += rng.normal(0, noise_rel * rngv, f.shape)
    return f.astype(np.float32)


def random_walk_1d(n=1 << 28, seed=1002, step=1e-2, spike_frac=0.01):
    """Workload 2 (HACC-like 1D): Gaussian random walk with step sigma 1e-2;
    1% of points (uniform, without replacement) replaced by spikes uniform in
    the walk's [min, max]."""
    rng = np.random.default_rng(seed)
    steps = rng.standard_normal(n, dtype=np.float32)
    steps *= np.float32(step)
    walk = np.cumsum(steps, dtype=np.float64).astype(np.float32)
    del steps
    lo, hi = float(walk.min()), float(walk.max())
    k = int(round(spike_frac * n))
    if k:
        idx = rng.choice(n, size=k, replace=False)
        walk[idx] = rng.uniform(lo, hi, k).astype(np.float32)
    return walk


def gaussian_random_field(shape, slope, seed, unit_variance=True):
    """Gaussian random field with isotropic power spectrum P(k) ~ k^slope,
    by filtering white noise in Fourier space."""
    fft, kw = _fft()
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shape).astype(np.float32)
    W = fft.rfftn(w, **kw)
    del w
    ks = [np.fft.fftfreq(s).astype(np.float32) for s in shape[:-1]] + [np.fft.rfftfreq(shape[-1]).astype(np.float32)]
    k2 = np.zeros(W.shape, np.float32)
    for ax, kk in enumerate(ks):
        sh = [1] * len(shape)
        sh[ax] = kk.size
        k2 += kk.reshape(sh) ** 2
    k2.flat[0] = 1.0
    amp = k2 ** np.float32(slope / 4.0)  # |k|^(slope/2)
    amp.flat[0] = 0.0
    W *= amp
    del amp, k2
    g = fft.irfftn(W, s=shape, **kw).astype(np.float32)
    if unit_variance:
        g -= g.mean()
        g /= g.std()
    return g


def grf_2d_batch(nfields=16, ny=1800, nx=3600, seed=1003, masked=(0, 5, 10, 15), mask_frac=0.2):
    """Workload 3 (CESM-ATM-like 2D): fields of a power-law -3 Gaussian random
    field, unit variance; the listed fields get ~20% of their area, as
    axis-aligned rectangles, set to the field minimum (near-zero regions of
    the paper's Table "nearzero")."""
    out = []
    rng = np.random.default_rng(seed)
    for i in range(nfields):
        g = gaussian_random_field((ny, nx), -3.0, seed * 100 + i)
        if i in masked:
            target = mask_frac * ny * nx
            m = np.zeros((ny, nx), bool)
            while m.sum() < target:
                h = int(rng.integers(ny // 10, ny // 3))
                w = int(rng.integers(nx // 10, nx // 3))
                y0 = int(rng.integers(0, ny - h))
                x0 = int(rng.integers(0, nx - w))
                m[y0:y0 + h, x0:x0 + w] = True
            g[m] = g.min()
        out.append(g)
    return out


def lognormal_3d(n=512, seed=1004, slope=-2.5, sigma=1.0):
    """Workload 4 (Nyx baryon_density-like): exp of a spectrum -2.5 Gaussian
    random field of unit variance."""
    g = gaussian_random_field((n, n, n), slope, seed)
    g *= np.float32(sigma)
    np.exp(g, out=g)
    return g


def serving_mix(count=256, seed=1005, min_bytes=256 << 10, max_bytes=512 << 20):
    """Workload 5: request descriptors (rank, shape, generator, rel eb, arrival
    time, kind) for the serving mix; sizes log-uniform, Poisson arrivals at
    200 requests/s, half compress and half decompress."""
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for i in range(count):
        rank = int(rng.integers(1, 4))
        nbytes = float(np.exp(rng.uniform(np.log(min_bytes), np.log(max_bytes))))
        n = max(1, int(nbytes // 4))
        if rank == 1:
            shape = (n,)
        elif rank == 2:
            a = int(round(np.sqrt(n)))
            shape = (max(1, n // a), a)
        else:
            a = int(round(n ** (1 / 3)))
            shape = (max(1, n // (a * a)), a, a)
        t += float(rng.exponential(1 / 200.0))
        reqs.append(dict(id=i, rank=rank, shape=shape, gen=int(rng.integers(1, 5)),
                         rel=float(rng.choice([1e-2, 1e-3, 1e-4])), arrival=t,
                         kind="compress" if rng.random() < 0.5 else "decompress"))
    return reqs


def small_cases():
    """Parity-test shapes: several tiles and a ragged tail in each rank."""
    return {
        "1d": (100003,),
        "2d": (181, 1037),
        "3d": (37, 41, 67),
    }


def field_for(kind, shape, seed):
    """A small field of the given rank with the character of workloads 1-4."""
    rng = np.random.default_rng(seed)
    if kind == "walk":
        return np.cumsum(rng.normal(0, 1e-2, shape[0])).astype(np.float32)
    if kind == "grf":
        return gaussian_random_field(shape, -3.0 if len(shape) == 2 else -2.5, seed)
    if kind == "lognormal":
        return np.exp(gaussian_random_field(shape, -2.5, seed))
    if kind == "sinus":
        grids = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
        f = np.zeros(shape)
        for _ in range(8):
            k = rng.integers(1, 9, len(shape))
            f += rng.uniform(0.5, 1) * np.sin(sum(2 * np.pi * kk * g / s for kk, g, s in zip(k, grids, shape))
                                              + rng.uniform(0, 2 * np.pi))
        f += rng.normal(0, 1e-3 * (f.max() - f.min()), shape)
        return f.astype(np.float32)
    raise ValueError(kind)


def field_on_device(kind, shape, seed, device):
    """The generators of field_for, computed with torch on `device` (for the
    serving mix, whose 256 fields of up to 512 MiB would take minutes on the
    host).  Seeded by a device generator, so the values differ from
    field_for's numpy stream but follow the same recipe: a Gaussian random
    walk (step 1e-2), a power-law Gaussian random field (slope -3 in 2D,
    -2.5 otherwise) of unit variance, its exponential, or a sum of 8
    random-phase sinusoids plus noise of 1e-3 of the range."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    n = 1
    for s in shape:
        n *= s
    if kind == "walk":
        steps = torch.randn(n, generator=g, device=device, dtype=torch.float32) * 1e-2
        return torch.cumsum(steps.double(), 0).float().reshape(shape)
    if kind in ("grf", "lognormal"):
        slope = -3.0 if (kind == "grf" and len(shape) == 2) else -2.5
        w = torch.randn(shape, generator=g, device=device, dtype=torch.float32)
        W = torch.fft.rfftn(w)
        del w
        k2 = torch.zeros(W.shape, device=device, dtype=torch.float32)
        for ax, s in enumerate(shape):
            kk = torch.fft.rfftfreq(s, device=device) if ax == len(shape) - 1 else torch.fft.fftfreq(s, device=device)
            sh = [1] * len(shape)
            sh[ax] = kk.numel()
            k2 += kk.float().reshape(sh) ** 2
        k2.view(-1)[0] = 1.0
        amp = k2 ** (slope / 4.0)
        amp.view(-1)[0] = 0.0
        W *= amp
        del amp, k2
        f = torch.fft.irfftn(W, s=shape)
        del W
        f = (f - f.mean()) / f.std()
        return torch.exp(f) if kind == "lognormal" else f.contiguous()
    if kind == "sinus":
        f = torch.zeros(shape, device=device, dtype=torch.float32)
        grids = torch.meshgrid(*[torch.arange(s, device=device, dtype=torch.float32) / s for s in shape],
                               indexing="ij")
        for _ in range(8):
            k = torch.randint(1, 9, (len(shape),), generator=g, device=device).float()
            a = 0.5 + 0.5 * torch.rand((), generator=g, device=device)
            ph = 2 * np.pi * torch.rand((), generator=g, device=device)
            arg = sum(kk * gg for kk, gg in zip(k, grids)) * (2 * np.pi) + ph
            f += a * torch.sin(arg)
        rng_ = f.max() - f.min()
        f += torch.randn(shape, generator=g, device=device) * (1e-3 * rng_)
        return f
    raise ValueError(kind)
