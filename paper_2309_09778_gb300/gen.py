"""Seeded synthetic input fields.

This module only draws inputs: it holds none of the compressor's arithmetic and
is shared, as input bits, by the CPU oracle tests and the CUDA path.

The paper evaluates on SEG-Y seismic volumes (Section VI.A), which are not
available here.  Smooth Gaussian random fields stand in for them: white noise
from numpy's Philox counter-based generator, shaped in Fourier space to a power
spectrum |k|^-beta (k = 0 mode removed), normalised to mean 0 and sd 1.  Values
are made log-normal in magnitude with an independent sign field, and exact
zeros fill the regions where a third field lies below a quantile, which gives
contiguous zero regions like muted seismic zones.
"""
from __future__ import annotations

import numpy as np


def grf(shape, beta: float, seed: int) -> np.ndarray:
    """Gaussian random field with power spectrum |k|^-beta, float64, mean 0, sd 1."""
    shape = tuple(int(s) for s in shape)
    rng = np.random.Generator(np.random.Philox(seed))
    white = rng.standard_normal(shape)
    spec = np.fft.rfftn(white)
    k2 = np.zeros(spec.shape)
    for ax, n in enumerate(shape):
        if ax == len(shape) - 1:
            f = np.fft.rfftfreq(n)
        else:
            f = np.fft.fftfreq(n)
        sl = [None] * len(shape)
        sl[ax] = slice(None)
        k2 = k2 + (f[tuple(sl)] ** 2)
    with np.errstate(divide="ignore"):
        amp = np.where(k2 > 0, k2 ** (-beta / 4.0), 0.0)
    g = np.fft.irfftn(spec * amp, s=shape, axes=tuple(range(len(shape))))
    g -= g.mean()
    sd = g.std()
    if sd > 0:
        g /= sd
    return g


def grf_device(shape, beta: float, seed: int, device):
    """grf() with the Fourier shaping done by torch on `device` (float64).

    The white noise is numpy's Philox draw, as in grf(); the FFTs run on the
    device so that the 512^3 workloads are made in seconds.  Returns a float64
    torch tensor on `device`, mean 0 and sd 1.
    """
    import torch
    shape = tuple(int(s) for s in shape)
    rng = np.random.Generator(np.random.Philox(seed))
    white = torch.from_numpy(rng.standard_normal(shape)).to(device)
    spec = torch.fft.rfftn(white)
    del white
    k2 = torch.zeros((), dtype=torch.float64, device=device)
    for ax, n in enumerate(shape):
        f = torch.fft.rfftfreq(n, dtype=torch.float64, device=device) if ax == len(shape) - 1 else \
            torch.fft.fftfreq(n, dtype=torch.float64, device=device)
        k2 = k2 + (f ** 2).reshape([-1 if a == ax else 1 for a in range(len(shape))])
    amp = torch.where(k2 > 0, k2.clamp_min(1e-300) ** (-beta / 4.0), torch.zeros_like(k2))
    spec *= amp
    del amp, k2
    g = torch.fft.irfftn(spec, s=shape, dim=tuple(range(len(shape))))
    del spec
    g -= g.mean()
    sd = g.std(correction=0)
    if sd > 0:
        g /= sd
    return g


def grf_torch_noise(shape, beta: float, seed: int, device):
    """Gaussian random field with spectrum |k|^-beta from torch's own seeded
    device generator (white noise drawn on the device; float64, mean 0, sd 1).
    Used for the many-field batch, where drawing the noise on the host would
    dominate; deterministic for a given seed, device type and torch version."""
    import torch
    shape = tuple(int(s) for s in shape)
    gen_ = torch.Generator(device=device)
    gen_.manual_seed(int(seed))
    white = torch.randn(shape, generator=gen_, dtype=torch.float64, device=device)
    spec = torch.fft.rfftn(white)
    del white
    k2 = torch.zeros((), dtype=torch.float64, device=device)
    for ax, n in enumerate(shape):
        f = torch.fft.rfftfreq(n, dtype=torch.float64, device=device) if ax == len(shape) - 1 else \
            torch.fft.fftfreq(n, dtype=torch.float64, device=device)
        k2 = k2 + (f ** 2).reshape([-1 if a == ax else 1 for a in range(len(shape))])
    spec *= torch.where(k2 > 0, k2.clamp_min(1e-300) ** (-beta / 4.0), torch.zeros_like(k2))
    g = torch.fft.irfftn(spec, s=shape, dim=tuple(range(len(shape))))
    del spec
    g -= g.mean()
    sd = g.std(correction=0)
    if sd > 0:
        g /= sd
    return g


def signed_lognormal_device(shape, beta: float, seed: int, device, log_scale: float = 2.0,
                            zero_frac: float = 0.05):
    """signed_lognormal() drawn entirely on the device (grf_torch_noise), float32 tensor."""
    import torch
    x = torch.exp(log_scale * grf_torch_noise(shape, beta, seed, device))
    x *= torch.where(grf_torch_noise(shape, beta, seed + 1, device) >= 0, 1.0, -1.0)
    if zero_frac > 0:
        g3 = grf_torch_noise(shape, beta, seed + 2, device).float()
        k = max(1, int(round(zero_frac * g3.numel())))
        thr = torch.kthvalue(g3.reshape(-1), k).values.item()
        x = torch.where(g3 < thr, torch.zeros_like(x), x)
    return x.to(torch.float32)


def density_velocity_pair(shape, device, seed_density: int = 0, seed_velocity: int = 3):
    """The 512^3-style pair: positive density exp(1.5 G), G with spectrum k^-2, and a
    signed velocity-like G with spectrum k^-4; float32 torch tensors on `device`."""
    import torch
    rho = torch.exp(1.5 * grf_device(shape, 2.0, seed_density, device)).to(torch.float32)
    vel = grf_device(shape, 4.0, seed_velocity, device).to(torch.float32)
    return rho, vel


def wide_range_device(shape, beta: float, seed: int, device, decades: float = 8.0, zero_frac: float = 0.01):
    """wide_range() on the device: |x| = 10^(decades G1 / max|G1|), sign of G2, exact zeros where
    G3 lies below its quantile; a float64 torch tensor on `device`."""
    import torch
    g1 = grf_device(shape, beta, seed, device)
    m = g1.abs().max()
    x = torch.pow(10.0, decades * g1 / (m if m > 0 else 1.0))
    del g1
    x *= torch.where(grf_device(shape, beta, seed + 1, device) >= 0, 1.0, -1.0)
    if zero_frac > 0:
        g3 = grf_device(shape, beta, seed + 2, device)
        k = max(1, int(round(zero_frac * g3.numel())))
        thr = torch.kthvalue(g3.reshape(-1).cpu(), k).values.item()
        x = torch.where(g3 < thr, torch.zeros_like(x), x)
    return x


def signed_lognormal(shape, beta: float, seed: int, log_scale: float = 2.0,
                     zero_frac: float = 0.05, dtype=np.float32) -> np.ndarray:
    """|x| = exp(log_scale * G1), sign from G2, exact zeros where G3 < its quantile."""
    g1 = grf(shape, beta, seed)
    g2 = grf(shape, beta, seed + 1)
    x = np.exp(log_scale * g1) * np.where(g2 >= 0, 1.0, -1.0)
    if zero_frac > 0:
        g3 = grf(shape, beta, seed + 2)
        thr = np.quantile(g3, zero_frac)
        x = np.where(g3 < thr, 0.0, x)
    return x.astype(dtype)


def positive_lognormal(shape, beta: float, seed: int, log_scale: float,
                       dtype=np.float32) -> np.ndarray:
    """Density-like positive field exp(log_scale * G)."""
    return np.exp(log_scale * grf(shape, beta, seed)).astype(dtype)


def signed_grf(shape, beta: float, seed: int, dtype=np.float32) -> np.ndarray:
    """Velocity-like signed field G itself."""
    return grf(shape, beta, seed).astype(dtype)


def wide_range(shape, beta: float, seed: int, decades: float = 8.0,
               zero_frac: float = 0.01, dtype=np.float64) -> np.ndarray:
    """|x| = 10^(decades * G1 / max|G1|), mixed sign, exact zeros (float64 workload)."""
    g1 = grf(shape, beta, seed)
    g2 = grf(shape, beta, seed + 1)
    m = np.abs(g1).max()
    x = np.power(10.0, decades * g1 / (m if m > 0 else 1.0)) * np.where(g2 >= 0, 1.0, -1.0)
    if zero_frac > 0:
        g3 = grf(shape, beta, seed + 2)
        thr = np.quantile(g3, zero_frac)
        x = np.where(g3 < thr, 0.0, x)
    return x.astype(dtype)


# Named workloads.  Sizes, spectra, value distributions and error bounds follow
# the evaluation plan: a small 64^3 single-precision case, a 100x500x500 case,
# a 512^3 density/velocity pair and a 256x384x384 double-precision case.
WORKLOADS = {
    "grf64_f32": dict(shape=(64, 64, 64), beta=3.0, seed=0, zero_frac=0.05, eb=1e-2),
    "grf100x500x500_f32": dict(shape=(100, 500, 500), beta=11.0 / 3.0, seed=0,
                               zero_frac=0.02, eb=1e-3),
}


def workload(name: str, shape=None) -> tuple[np.ndarray, float]:
    """Return (field, eb_rel) for a named workload, optionally at a smaller shape."""
    w = WORKLOADS[name]
    shp = w["shape"] if shape is None else shape
    x = signed_lognormal(shp, w["beta"], w["seed"], 2.0, w["zero_frac"])
    return x, w["eb"]
