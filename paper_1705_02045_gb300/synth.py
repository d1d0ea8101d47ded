"""Seeded synthetic images shared by the tests, the benchmark and the CPU oracle.

This module only draws inputs; it holds none of the Euler-characteristic
arithmetic. Every generator is deterministic for a given seed (numpy PCG64 via
``default_rng``), so the GPU path and the oracle consume the same bytes.

Recipes (the paper's own images are not distributed with it; these stand in
for them with the shapes, value ranges and smoothness of its workloads):

* ``uniform_u8``    i.i.d. uniform 0..255 (the paper's "random8" images).
* ``smooth_u8``     white noise N(0,1) -> separable Gaussian, truncated at 4
                    sigma, reflect border -> linear requantisation of
                    [min, max] to 0..255, rounded half-to-even.
* ``two_phase_u16`` Gaussian random field (as above, normalised by the
                    filter's theoretical standard deviation) thresholded at the
                    analytic 40th percentile of N(0,1); voxels below the
                    threshold ~ N(3000, 400), the rest ~ N(11000, 900), i.i.d.,
                    rounded half-to-even, clipped to 0..16383 (14-bit micro-CT
                    stand-in).
* ``grf_f32``       normalised Gaussian random field, float32, left continuous.
* ``request_mix``   shapes and dtypes of a mixed request stream.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 1705020450

# Phi^{-1}(0.4): the 40th percentile of the standard normal distribution.
Z_040 = -0.2533471031357997


def uniform_u8(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=tuple(shape), dtype=np.uint8)


def uniform_int(shape, high: int, seed: int, dtype=np.uint16) -> np.ndarray:
    """i.i.d. uniform integers in [0, high)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, high, size=tuple(shape), dtype=np.int64).astype(dtype)


def _gaussian_field(shape, sigma: float, seed: int) -> np.ndarray:
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(size=tuple(shape), dtype=np.float32)
    return gaussian_filter(noise, sigma=sigma, mode="reflect", truncate=4.0)


def _filter_std(sigma: float, ndim: int) -> float:
    """Standard deviation of unit white noise after the truncated, normalised
    Gaussian filter (interior of the image): prod over axes of ||w||_2."""
    r = int(4.0 * sigma + 0.5)
    x = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-0.5 * (x / sigma) ** 2)
    w /= w.sum()
    return float(np.sqrt(np.sum(w * w)) ** ndim)


def requantise(x: np.ndarray, top: int, dtype) -> np.ndarray:
    lo, hi = float(x.min()), float(x.max())
    scale = top / (hi - lo) if hi > lo else 0.0
    return np.rint((x.astype(np.float64) - lo) * scale).astype(dtype)


def smooth_u8(shape, sigma: float, seed: int) -> np.ndarray:
    return requantise(_gaussian_field(shape, sigma, seed), 255, np.uint8)


def smooth_int(shape, sigma: float, top: int, seed: int, dtype) -> np.ndarray:
    """Smoothed Gaussian field requantised linearly to 0..top."""
    return requantise(_gaussian_field(shape, sigma, seed), top, dtype)


def two_phase_u16(shape, sigma: float, seed: int) -> np.ndarray:
    field = _gaussian_field(shape, sigma, seed) / _filter_std(sigma, len(shape))
    rng = np.random.default_rng(seed + 1)
    low = rng.normal(3000.0, 400.0, size=field.shape)
    high = rng.normal(11000.0, 900.0, size=field.shape)
    v = np.where(field < Z_040, low, high)
    return np.clip(np.rint(v), 0, 16383).astype(np.uint16)


def grf_f32(shape, sigma: float, seed: int) -> np.ndarray:
    field = _gaussian_field(shape, sigma, seed) / _filter_std(sigma, len(shape))
    return field.astype(np.float32)


def _gauss_weights(sigma: float):
    r = int(4.0 * sigma + 0.5)
    x = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-0.5 * (x / sigma) ** 2)
    return (w / w.sum()).astype(np.float32), r


def smooth_int_torch(shape, sigma: float, top, seed: int, device="cuda"):
    """The smoothed-field recipe (white noise -> separable Gaussian, truncated
    at 4 sigma, reflect border -> linear requantisation to 0..top) computed
    with torch on `device`, for workloads too large to generate with scipy in
    a benchmark run. Returns an int32 tensor on `device` (top = None: the
    float field before requantisation). Deterministic for a given seed, device
    type and torch version (not bit-identical to the numpy generators)."""
    import torch
    import torch.nn.functional as F

    g = torch.Generator(device=device).manual_seed(int(seed))
    x = torch.randn(tuple(shape), generator=g, device=device, dtype=torch.float32)
    w, r = _gauss_weights(sigma)
    wt = torch.from_numpy(w).to(device).view(1, 1, -1)
    for axis in range(x.dim()):
        n = x.shape[axis]
        if n <= 1:
            continue
        # border extension as scipy's "reflect" (d c b a | a b c d | d c b a)
        p = np.arange(-r, n + r)
        while np.any((p < 0) | (p >= n)):
            p = np.where(p < 0, -p - 1, p)
            p = np.where(p >= n, 2 * n - p - 1, p)
        idx = torch.from_numpy(p).to(device)
        y = x.movedim(axis, -1).contiguous()
        lead = y.shape[:-1]
        y = y.reshape(-1, n)
        out = torch.empty_like(y)
        for r0 in range(0, y.shape[0], 32768):
            blk = y[r0:r0 + 32768].index_select(1, idx).unsqueeze(1)
            out[r0:r0 + 32768] = F.conv1d(blk, wt).squeeze(1)
        x = out.reshape(*lead, n).movedim(-1, axis)
    if top is None:
        return x
    lo, hi = x.min(), x.max()
    scale = top / (hi - lo) if float(hi - lo) > 0 else 0.0
    return torch.round((x - lo) * scale).to(torch.int32)


def grf_f32_torch(shape, sigma: float, seed: int, device="cuda"):
    """grf_f32's recipe (normalised Gaussian random field, float32) computed
    with torch on `device`."""
    x = smooth_int_torch(shape, sigma, None, seed, device)
    return x / _filter_std(sigma, len(shape))


def two_phase_u16_slabs(shape, sigma: float, seed: int, slab: int, device="cuda"):
    """The two-phase 14-bit recipe for volumes too large for host-side
    generation, one z-slab at a time on the GPU (yields (z0, uint16 host
    array)). Each plane's noise is drawn from its own seeded generator
    (seed + plane index), and the z-filter of a slab reads sigma * 4 planes
    of noise on either side (reflected at the volume's ends), so the field is
    the same as filtering the whole volume at once."""
    import torch
    import torch.nn.functional as F

    nz, ny, nx = shape
    w, r = _gauss_weights(sigma)
    wt = torch.from_numpy(w).to(device)
    std = _filter_std(sigma, 3)

    def noise_plane(z):
        zz = z
        while zz < 0 or zz >= nz:  # reflect like scipy
            zz = -zz - 1 if zz < 0 else 2 * nz - zz - 1
        g = torch.Generator(device=device).manual_seed(int(seed) * 100003 + zz)
        return torch.randn((ny, nx), generator=g, device=device, dtype=torch.float32)

    def filt_last(x, n):
        p = np.arange(-r, n + r)
        while np.any((p < 0) | (p >= n)):
            p = np.where(p < 0, -p - 1, p)
            p = np.where(p >= n, 2 * n - p - 1, p)
        idx = torch.from_numpy(p).to(device)
        lead = x.shape[:-1]
        y = x.reshape(-1, n)
        out = torch.empty_like(y)
        for r0 in range(0, y.shape[0], 32768):
            out[r0:r0 + 32768] = F.conv1d(y[r0:r0 + 32768].index_select(1, idx).unsqueeze(1),
                                          wt.view(1, 1, -1)).squeeze(1)
        return out.reshape(*lead, n)

    for z0 in range(0, nz, slab):
        z1 = min(z0 + slab, nz)
        planes = []
        for z in range(z0 - r, z1 + r):  # x and y filtered noise planes
            p = filt_last(noise_plane(z), nx)
            p = filt_last(p.t().contiguous(), ny).t()
            planes.append(p)
        vol = torch.stack(planes)  # (z1 - z0 + 2r, ny, nx)
        field = torch.zeros((z1 - z0, ny, nx), device=device, dtype=torch.float32)
        for k in range(2 * r + 1):
            field += float(w[k]) * vol[k:k + (z1 - z0)]
        del vol, planes
        field /= std
        g = torch.Generator(device=device).manual_seed(int(seed) * 7919 + z0)
        low = torch.randn(field.shape, generator=g, device=device) * 400.0 + 3000.0
        high = torch.randn(field.shape, generator=g, device=device) * 900.0 + 11000.0
        v = torch.where(field < Z_040, low, high)
        out = torch.clamp(torch.round(v), 0, 16383).to(torch.int16)
        yield z0, out.cpu().numpy().view(np.uint16)


def request_mix(n: int, seed: int):
    """Shapes/dtypes of a mixed request stream: 2D:3D = 50:50, side
    log-uniform in [64, 2048] (2D) or [32, 384] (3D), isotropic; dtype uint8
    (60 %) or 14-bit uint16 (40 %). Returns a list of (shape, dtype, bins)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        if rng.random() < 0.5:
            s = int(round(math.exp(rng.uniform(math.log(64), math.log(2048)))))
            shape = (s, s)
        else:
            s = int(round(math.exp(rng.uniform(math.log(32), math.log(384)))))
            shape = (s, s, s)
        if rng.random() < 0.6:
            out.append((shape, np.uint8, 256))
        else:
            out.append((shape, np.uint16, 16384))
    return out
