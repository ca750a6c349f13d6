"""Seeded synthetic fields shaped like the paper's workloads (Table 1).

The paper evaluates on NYX (cosmology, 3D), CESM-ATM (climate, 2D 1800x3600)
and Hurricane ISABELA (3D 100x500x500); none of those data sets is available
here, so these generators stand in for them with the same shapes and the
value structure the evaluation depends on (smooth multi-scale fields, heavy
tails, constant regions, spikes).  This module holds none of the compression
arithmetic: it only draws numbers.  It is shared by the tests, the benchmark
and the smoke check, and is the only code the CUDA path and the oracle share.

All fields are generated in FP64 (numpy FFT, or torch FFT on a given device
for the large 3D cases) and cast to float32 at the end.
"""
from __future__ import annotations

import math

import numpy as np

PSNR_SWEEP_2D = (40.0, 60.0, 80.0, 100.0, 120.0)


def _kgrid(shape, stretch=None):
    """|k| on the rfftn grid (cycles per sample); stretch[i] divides axis i's k."""
    axes = []
    for i, n in enumerate(shape):
        k = np.fft.rfftfreq(n) if i == len(shape) - 1 else np.fft.fftfreq(n)
        if stretch is not None:
            k = k / stretch[i]
        axes.append(k)
    grids = np.meshgrid(*axes, indexing="ij", sparse=True)
    k2 = sum(g * g for g in grids)
    return np.sqrt(k2)


def grf(shape, alpha: float, seed: int, stretch=None, rng=None) -> np.ndarray:
    """Gaussian random field with power spectrum P(k) ~ k^-alpha (k=0 zeroed),
    zero mean, unit standard deviation, float64."""
    rng = rng if rng is not None else np.random.default_rng(seed)
    white = rng.standard_normal(shape)
    spec = np.fft.rfftn(white)
    k = _kgrid(shape, stretch)
    with np.errstate(divide="ignore"):
        amp = np.where(k > 0, k ** (-alpha / 2.0), 0.0)
    f = np.fft.irfftn(spec * amp, s=shape, axes=list(range(len(shape))))
    f -= f.mean()
    sd = f.std()
    return f / sd if sd > 0 else f


def grf_torch(shape, alpha: float, seed: int, device, stretch=None):
    """Same construction with torch on `device` (for 512^3 fields); returns a
    float64 torch tensor.  Seeded by a torch.Generator on that device."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    white = torch.randn(shape, generator=g, device=device, dtype=torch.float64)
    spec = torch.fft.rfftn(white)
    del white
    k2 = None
    for i, n in enumerate(shape):
        if i == len(shape) - 1:
            k = torch.fft.rfftfreq(n, device=device, dtype=torch.float64)
        else:
            k = torch.fft.fftfreq(n, device=device, dtype=torch.float64)
        if stretch is not None:
            k = k / stretch[i]
        view = [1] * len(shape)
        view[i] = -1
        k = k.reshape(view) ** 2
        k2 = k if k2 is None else k2 + k
    kk = torch.sqrt(k2)
    amp = torch.where(kk > 0, kk.clamp_min(1e-300) ** (-alpha / 2.0), torch.zeros_like(kk))
    spec *= amp
    del kk, k2, amp
    f = torch.fft.irfftn(spec, s=shape)
    del spec
    f -= f.mean()
    sd = f.std()
    if sd > 0:
        f /= sd
    return f


def rescale(f: np.ndarray, lo: float, hi: float) -> np.ndarray:
    fmin, fmax = float(f.min()), float(f.max())
    if fmax == fmin:
        return np.full_like(f, lo)
    return (f - fmin) / (fmax - fmin) * (hi - lo) + lo


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def single_2d(n: int = 512, seed: int = 0) -> np.ndarray:
    """One 512x512 field: isotropic GRF, P(k) ~ k^-3, rescaled to [-1, 1]."""
    return rescale(grf((n, n), 3.0, seed), -1.0, 1.0).astype(np.float32)


def climate_batch(count: int = 24, ny: int = 1800, nx: int = 3600, seed: int = 1, device=None):
    """ATM-like batch: per field alpha ~ U[2,4], value = offset + scale * g with
    g the GRF rescaled to [-1, 1], scale = 10^U(-3,5), offset = +-10^U(-3,5);
    round(5% of count) fields get a seeded rectangle held at the field minimum.
    Returns (list of float32 arrays, list of per-field metadata dicts); with
    `device` the GRFs are drawn with torch there and the fields are float32
    torch tensors on that device (same recipe, different random stream)."""
    if device is not None:
        return _climate_batch_torch(count, ny, nx, seed, device)
    rng = np.random.default_rng(seed)
    n_const = int(round(0.05 * count))
    const_ids = set(rng.choice(count, size=n_const, replace=False).tolist()) if n_const else set()
    fields, meta = [], []
    for i in range(count):
        alpha = float(rng.uniform(2.0, 4.0))
        scale = 10.0 ** float(rng.uniform(-3.0, 5.0))
        offset = (1.0 if rng.uniform() < 0.5 else -1.0) * 10.0 ** float(rng.uniform(-3.0, 5.0))
        fseed = int(rng.integers(0, 2**31 - 1))
        g = rescale(grf((ny, nx), alpha, fseed), -1.0, 1.0)
        f = offset + scale * g
        rect = None
        if i in const_ids:
            h = int(rng.integers(ny // 10, ny // 3))
            w = int(rng.integers(nx // 10, nx // 3))
            y0 = int(rng.integers(0, ny - h))
            x0 = int(rng.integers(0, nx - w))
            f[y0:y0 + h, x0:x0 + w] = f.min()
            rect = (y0, x0, h, w)
        fields.append(f.astype(np.float32))
        meta.append(dict(alpha=alpha, scale=scale, offset=offset, seed=fseed, const_rect=rect))
    return fields, meta


def _climate_batch_torch(count, ny, nx, seed, device):
    import torch
    rng = np.random.default_rng(seed)
    n_const = int(round(0.05 * count))
    const_ids = set(rng.choice(count, size=n_const, replace=False).tolist()) if n_const else set()
    fields, meta = [], []
    for i in range(count):
        alpha = float(rng.uniform(2.0, 4.0))
        scale = 10.0 ** float(rng.uniform(-3.0, 5.0))
        offset = (1.0 if rng.uniform() < 0.5 else -1.0) * 10.0 ** float(rng.uniform(-3.0, 5.0))
        fseed = int(rng.integers(0, 2**31 - 1))
        g = grf_torch((ny, nx), alpha, fseed, device)
        gmin, gmax = g.min(), g.max()
        g = (g - gmin) / (gmax - gmin) * 2.0 - 1.0
        f = offset + scale * g
        rect = None
        if i in const_ids:
            h = int(rng.integers(ny // 10, ny // 3))
            w = int(rng.integers(nx // 10, nx // 3))
            y0 = int(rng.integers(0, ny - h))
            x0 = int(rng.integers(0, nx - w))
            f[y0:y0 + h, x0:x0 + w] = f.min()
            rect = (y0, x0, h, w)
        fields.append(f.to(torch.float32).contiguous())
        meta.append(dict(alpha=alpha, scale=scale, offset=offset, seed=fseed, const_rect=rect))
        del g, f
    return fields, meta


def mixed_psnr(i: int, sweep=PSNR_SWEEP_2D) -> float:
    """Target PSNR of field i in the mixed sweep run: sweep[i mod len(sweep)]."""
    return float(sweep[i % len(sweep)])


def hurricane_batch(count: int = 13, nz: int = 100, ny: int = 500, nx: int = 500, seed: int = 2,
                    device=None):
    """Hurricane-like batch: anisotropic GRFs (horizontal correlation length 4x
    the vertical one; z is the slowest, vertical axis), field 0 plus a smooth
    vortex-shaped mean, two fields with 0.1% of points spiked to 50x the std.
    Returns (fields, meta); target PSNRs are 30..120 dB step 10 (psnr_i).
    With `device` the fields are drawn with torch there and returned as
    float32 torch tensors on that device (same recipe, different random
    stream)."""
    if device is not None:
        return _hurricane_batch_torch(count, nz, ny, nx, seed, device)
    rng = np.random.default_rng(seed)
    spike_ids = set(rng.choice(np.arange(1, count), size=min(2, count - 1), replace=False).tolist()) \
        if count > 1 else set()
    fields, meta = [], []
    for i in range(count):
        fseed = int(rng.integers(0, 2**31 - 1))
        g = grf((nz, ny, nx), 3.0, fseed, stretch=(4.0, 1.0, 1.0))
        if i == 0:
            zz, yy, xx = np.meshgrid(np.linspace(0, 1, nz), np.linspace(-1, 1, ny),
                                     np.linspace(-1, 1, nx), indexing="ij", sparse=True)
            r = np.sqrt(xx * xx + yy * yy) / 0.3
            g = g + 5.0 * r * np.exp(1.0 - r) * (1.0 - 0.5 * zz)
        spikes = 0
        if i in spike_ids:
            sd = float(g.std())
            m = rng.uniform(size=g.shape) < 1e-3
            g = np.where(m, g + 50.0 * sd, g)
            spikes = int(m.sum())
        fields.append(g.astype(np.float32))
        meta.append(dict(seed=fseed, vortex=(i == 0), spikes=spikes, psnr=30.0 + 10.0 * (i % 10)))
    return fields, meta


def _hurricane_batch_torch(count, nz, ny, nx, seed, device):
    import torch
    rng = np.random.default_rng(seed)
    spike_ids = set(rng.choice(np.arange(1, count), size=min(2, count - 1), replace=False).tolist()) \
        if count > 1 else set()
    fields, meta = [], []
    for i in range(count):
        fseed = int(rng.integers(0, 2**31 - 1))
        g = grf_torch((nz, ny, nx), 3.0, fseed, device, stretch=(4.0, 1.0, 1.0))
        if i == 0:
            zz = torch.linspace(0, 1, nz, device=device, dtype=torch.float64).reshape(nz, 1, 1)
            yy = torch.linspace(-1, 1, ny, device=device, dtype=torch.float64).reshape(1, ny, 1)
            xx = torch.linspace(-1, 1, nx, device=device, dtype=torch.float64).reshape(1, 1, nx)
            r = torch.sqrt(xx * xx + yy * yy) / 0.3
            g = g + 5.0 * r * torch.exp(1.0 - r) * (1.0 - 0.5 * zz)
        spikes = 0
        if i in spike_ids:
            sd = float(g.std())
            gen = torch.Generator(device=device)
            gen.manual_seed(fseed + 1)
            m = torch.rand(g.shape, generator=gen, device=device, dtype=torch.float64) < 1e-3
            g = torch.where(m, g + 50.0 * sd, g)
            spikes = int(m.sum().item())
        fields.append(g.to(torch.float32).contiguous())
        meta.append(dict(seed=fseed, vortex=(i == 0), spikes=spikes, psnr=30.0 + 10.0 * (i % 10)))
        del g
    return fields, meta


def cosmology_fields(n: int = 512, seed: int = 3, device=None):
    """NYX-like set of 6 n^3 fields: 2 densities exp(G) (G: P ~ k^-2, sigma 2),
    3 velocity components (P ~ k^-3), 1 temperature exp(0.5 G).  With `device`
    the fields are generated there with torch and returned as float32 torch
    tensors on that device; otherwise numpy float32 arrays."""
    rng = np.random.default_rng(seed)
    seeds = [int(s) for s in rng.integers(0, 2**31 - 1, size=6)]
    kinds = ["density", "density", "velocity", "velocity", "velocity", "temperature"]
    out = []
    for kind, s in zip(kinds, seeds):
        if device is not None:
            import torch
            alpha = 3.0 if kind == "velocity" else 2.0
            g = grf_torch((n, n, n), alpha, s, device)
            if kind == "density":
                g = torch.exp(2.0 * g)
            elif kind == "temperature":
                g = torch.exp(0.5 * 2.0 * g)
            out.append(g.to(torch.float32))
            del g
        else:
            alpha = 3.0 if kind == "velocity" else 2.0
            g = grf((n, n, n), alpha, s)
            if kind == "density":
                g = np.exp(2.0 * g)
            elif kind == "temperature":
                g = np.exp(0.5 * 2.0 * g)
            out.append(g.astype(np.float32))
    return out, kinds


def smooth_3d(shape, seed: int) -> np.ndarray:
    """Small isotropic 3D GRF (P ~ k^-3) rescaled to [-1, 1], for tests."""
    return rescale(grf(shape, 3.0, seed), -1.0, 1.0).astype(np.float32)


def smooth_1d(n: int, seed: int) -> np.ndarray:
    """1D GRF (P ~ k^-2) rescaled to [-1, 1]."""
    return rescale(grf((n,), 2.0, seed), -1.0, 1.0).astype(np.float32)


def uniform_noise(shape, seed: int, lo=-1.0, hi=1.0) -> np.ndarray:
    """White noise: a field with no spatial correlation (worst case for the
    predictor, widest code alphabet)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=shape).astype(np.float32)


def psnr_sweep_3d(i: int) -> float:
    return 30.0 + 10.0 * (i % 10)


def nbytes(shape) -> int:
    return 4 * int(math.prod(shape))
