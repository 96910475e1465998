"""Seeded synthetic fields shaped like the paper's scientific workloads.

The paper evaluates on NYX, LETKF, Miranda, Hurricane ISABEL and JHTDB
(Sec. 7.1, Table "Datasets"); none of them is available here, so these seeded
generators stand in for them.  This module holds no part of the refactoring
method: it only makes input arrays, and both the CUDA path and the CPU oracle
consume the same arrays.  Every random draw comes from a CPU ``torch.Generator``
so that a given seed gives the same parameters and noise on any device; the
optional ``device`` only moves the arithmetic (the spectral filter's FFT) to the
GPU for large fields.  ``device_noise=True`` draws the noise with a generator on
``device`` instead (much faster for benchmark-sized fields; reproducible on the
same device type and PyTorch version only).

* ``blobs``: sum of Gaussian blobs a*exp(-|x-c|^2 / (2 w^2)), centres uniform
  in the box, widths uniform in [4, 16] cells (scaled with the box for small
  boxes), amplitudes N(0, 1), plus N(0, 1e-3^2) noise.
* ``spectral``: Gaussian random field with isotropic power spectrum
  P(k) ~ |k|^(-11/3) (integer wavenumbers, k = 0 removed), rescaled to [-1, 1].
* ``spectral_trend``: ``spectral`` plus 0.5 sin(2 pi x / L_x) cos(2 pi y / L_y).
"""
import math

import torch


def _gen(seed, device="cpu"):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _normal(shape, seed_gen, seed, dtype, device, device_noise):
    if device_noise and str(device) != "cpu":
        return torch.randn(shape, generator=_gen(seed + 0x5EED, device), dtype=dtype, device=device)
    return torch.randn(shape, generator=seed_gen, dtype=dtype).to(device)


def blobs(shape, seed=0, n_blobs=8, width=(4.0, 16.0), noise=1e-3, dtype=torch.float32,
          device="cpu", device_noise=False):
    """Sum of ``n_blobs`` Gaussian blobs plus white noise on a (nz, ny, nx) grid."""
    shape = tuple(int(s) for s in shape)
    g = _gen(seed)
    nd = len(shape)
    centres = torch.rand((n_blobs, nd), generator=g, dtype=torch.float64) * torch.tensor(
        shape, dtype=torch.float64)
    scale = min(1.0, min(shape) / 64.0) if min(shape) > 1 else 1.0
    widths = (width[0] + (width[1] - width[0]) * torch.rand(n_blobs, generator=g,
                                                            dtype=torch.float64)) * max(scale, 0.25)
    amps = torch.randn(n_blobs, generator=g, dtype=torch.float64)
    f = _normal(shape, g, seed, torch.float64, device, device_noise) * noise
    axes = [torch.arange(s, dtype=torch.float64, device=device) for s in shape]
    for b in range(n_blobs):
        r2 = None
        for d in range(nd):
            dd = (axes[d] - float(centres[b, d])) ** 2
            view = [1] * nd
            view[d] = shape[d]
            dd = dd.view(view)
            r2 = dd if r2 is None else r2 + dd
        f = f + float(amps[b]) * torch.exp(-r2 / (2.0 * float(widths[b]) ** 2))
    return f.to(dtype).contiguous()


def _spectral_raw(shape, seed, slope, device, work_dtype, device_noise=False):
    g = _gen(seed)
    white = _normal(shape, g, seed, work_dtype, device, device_noise)
    spec = torch.fft.rfftn(white)
    del white
    ks = []
    nd = len(shape)
    for d, n in enumerate(shape):
        if d == nd - 1:
            k = torch.arange(n // 2 + 1, device=device, dtype=work_dtype)
        else:
            k = torch.fft.fftfreq(n, d=1.0 / n, device=device).to(work_dtype)
        view = [1] * nd
        view[d] = k.numel()
        ks.append((k * k).view(view))
    k2 = ks[0]
    for t in ks[1:]:
        k2 = k2 + t
    amp = torch.where(k2 > 0, k2.clamp_min(1e-30) ** (slope / 4.0), torch.zeros_like(k2))
    spec = spec * amp
    del amp, k2
    f = torch.fft.irfftn(spec, s=shape)
    return f


def _rescale(f):
    lo, hi = f.min(), f.max()
    return 2.0 * (f - lo) / (hi - lo) - 1.0


def spectral(shape, seed=2, slope=-11.0 / 3.0, dtype=torch.float32, device="cpu",
             device_noise=False):
    """Isotropic P(k) ~ k^slope Gaussian random field, rescaled to [-1, 1]."""
    shape = tuple(int(s) for s in shape)
    work = torch.float64 if dtype == torch.float64 else torch.float32
    f = _rescale(_spectral_raw(shape, seed, slope, device, work, device_noise))
    return f.to(dtype).contiguous()


def spectral_trend(shape, seed=3, slope=-11.0 / 3.0, dtype=torch.float64, device="cpu",
                   device_noise=False):
    """``spectral`` plus the smooth trend 0.5 sin(2 pi x/L_x) cos(2 pi y/L_y)."""
    shape = tuple(int(s) for s in shape)
    f = spectral(shape, seed=seed, slope=slope, dtype=torch.float64, device=device,
                 device_noise=device_noise)
    ny, nx = shape[-2], shape[-1]
    x = torch.arange(nx, dtype=torch.float64, device=device) * (2.0 * math.pi / nx)
    y = torch.arange(ny, dtype=torch.float64, device=device) * (2.0 * math.pi / ny)
    trend = 0.5 * torch.sin(x).view(1, 1, nx) * torch.cos(y).view(1, ny, 1)
    return (f + trend).to(dtype).contiguous()


def batch_sizes(count=256, lo=32, hi=256, seed=1):
    """Per-axis sizes drawn log-uniform in [lo, hi] (non-powers of two allowed)."""
    g = _gen(seed)
    u = torch.rand((count, 3), generator=g, dtype=torch.float64)
    sizes = torch.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))).round().to(torch.int64)
    return [tuple(int(v) for v in row) for row in sizes.clamp(lo, hi)]


def batch_field(i, shape, seed=1, device="cpu", device_noise=False):
    """i-th field of the batched workload: alternating blobs / spectral generators."""
    if i % 2 == 0:
        return blobs(shape, seed=seed * 100003 + i, device=device, device_noise=device_noise)
    return spectral(shape, seed=seed * 100003 + i, device=device, device_noise=device_noise)


def velocity_triplet(shape, seed=5, device="cpu", device_noise=False):
    """(vx, vy, vz), each an independent spectral field on `shape` (an int: a cube)."""
    if isinstance(shape, int):
        shape = (shape, shape, shape)
    return tuple(spectral(shape, seed=seed * 7 + c, device=device, device_noise=device_noise)
                 for c in range(3))
