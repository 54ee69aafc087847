"""Seeded synthetic fields shaped like the simulation outputs that MGARD+ is
evaluated on (Section 6.1, Table 2: Hurricane 100x500x500, NYX 512^3, ...).

The datasets themselves are not available, so every workload is generated
from a seed.  This module holds only input generation (random numbers, FFT
filtering, coordinates); it contains none of the decomposition arithmetic and
is the one module shared by the tests, the benchmark and the oracle-based
checks.  Pure numpy/scipy: no GPU is needed.
"""
from __future__ import annotations

import os

import numpy as np

__all__ = [
    "uniform_coords", "geometric_coords", "sinusoid_field", "grf_field",
    "front_field", "batched_shapes", "multilinear_field",
]

SEED_TINY = 2010058721
SEED_LARGE = 2010058722
SEED_NONUNIFORM = 2010058723
SEED_BATCHED = 2010058724
SEED_SERVING = 2010058725


def uniform_coords(n: int) -> np.ndarray:
    """``n`` equispaced coordinates on [0, 1]."""
    return np.linspace(0.0, 1.0, n)


def geometric_coords(n: int, ratio: float = 1.03) -> np.ndarray:
    """``n`` coordinates on [0, 1] whose spacings grow geometrically:
    ``D_k = D_0 * ratio**k``, normalised so the last coordinate is 1."""
    d = ratio ** np.arange(n - 1, dtype=np.float64)
    x = np.concatenate([[0.0], np.cumsum(d)])
    return x / x[-1]


def _unit_grid(dims, coords=None):
    if coords is None:
        coords = [uniform_coords(n) for n in dims]
    return np.meshgrid(*coords, indexing="ij", sparse=True)


def _ball_vectors(rng, count, ndim, radius):
    out = []
    while len(out) < count:
        k = rng.uniform(-radius, radius, size=ndim)
        if np.linalg.norm(k) <= radius:
            out.append(k)
    return np.array(out)


def sinusoid_field(dims, seed: int = SEED_TINY, n_modes: int = 4,
                   kmax: float = 8.0, noise: float = 1e-3,
                   dtype=np.float64) -> np.ndarray:
    """Sum of ``n_modes`` sinusoids ``a sin(2 pi k.x + phi)`` on [0,1]^d with
    real wavevectors uniform in the ball ``|k| <= kmax``, amplitudes
    U(0.5, 1), phases U(0, 2 pi), plus N(0, noise) white noise."""
    rng = np.random.default_rng(seed)
    ndim = len(dims)
    ks = _ball_vectors(rng, n_modes, ndim, kmax)
    amps = rng.uniform(0.5, 1.0, size=n_modes)
    phis = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    X = _unit_grid(dims)
    u = np.zeros(tuple(dims), dtype=np.float64)
    for k, a, p in zip(ks, amps, phis):
        arg = p + sum(2.0 * np.pi * k[d] * X[d] for d in range(ndim))
        u += a * np.sin(arg)
    u += rng.normal(0.0, noise, size=tuple(dims))
    return u.astype(dtype)


def grf_field(dims, seed: int = SEED_LARGE, slope: float = -5.0 / 3.0,
              dtype=np.float32) -> np.ndarray:
    """Gaussian random field with a shell-summed power spectrum
    ``E(k) ~ k^slope`` (Kolmogorov -5/3), made by filtering white noise in
    Fourier space in FP64 (per-mode amplitude ``|k|^((slope - d + 1)/2)``,
    mean removed) and scaling to unit variance."""
    from scipy import fft as sfft
    dims = tuple(int(n) for n in dims)
    ndim = len(dims)
    rng = np.random.default_rng(seed)
    white = rng.standard_normal(size=dims)
    workers = os.cpu_count() or 1
    spec = sfft.rfftn(white, workers=workers)
    del white
    k2 = None
    for d, n in enumerate(dims):
        f = (np.fft.rfftfreq(n) if d == ndim - 1 else np.fft.fftfreq(n)) * n
        shape = [1] * ndim
        shape[d] = len(f)
        term = (f.astype(np.float64) ** 2).reshape(shape)
        k2 = term if k2 is None else k2 + term
    with np.errstate(divide="ignore"):
        amp = np.where(k2 > 0, k2 ** ((slope - ndim + 1) / 4.0), 0.0)
    spec *= amp
    del amp, k2
    u = sfft.irfftn(spec, s=dims, workers=workers)
    del spec
    u -= u.mean()
    u /= u.std()
    return u.astype(dtype)


def grf_field_device(dims, seed: int, device="cuda", slope: float = -5.0 / 3.0):
    """The k^-5/3 field recipe of ``grf_field`` generated on a CUDA device
    (torch's seeded normal generator and FFTs in FP64), FP32 result: the
    input generator of the batched and serving workloads, where hundreds of
    fields are needed.  Its white noise is torch's, not numpy's, so the
    values differ from ``grf_field`` for the same seed."""
    import torch
    dims = tuple(int(n) for n in dims)
    ndim = len(dims)
    g = torch.Generator(device=device).manual_seed(int(seed))
    white = torch.randn(dims, generator=g, device=device, dtype=torch.float64)
    spec = torch.fft.rfftn(white)
    del white
    k2 = None
    for d, n in enumerate(dims):
        f = (torch.fft.rfftfreq(n, device=device) if d == ndim - 1
             else torch.fft.fftfreq(n, device=device)).double() * n
        shape = [1] * ndim
        shape[d] = f.numel()
        term = (f ** 2).reshape(shape)
        k2 = term if k2 is None else k2 + term
    amp = torch.where(k2 > 0, k2.clamp_min(1e-300) ** ((slope - ndim + 1) / 4.0),
                      torch.zeros_like(k2))
    spec *= amp
    u = torch.fft.irfftn(spec, s=dims)
    del spec
    u -= u.mean()
    u /= u.std()
    return u.float()


def front_field(dims, coords, seed: int = SEED_NONUNIFORM, n_modes: int = 3,
                width_cells: float = 5.0, dtype=np.float32) -> np.ndarray:
    """Smooth sinusoid sum plus a sharp ``tanh`` front across the diagonal
    ``p = (i + j + k)/sqrt(d)`` in index units, ``width_cells`` cells wide and
    centred on the grid centre (the non-uniform-grid workload)."""
    rng = np.random.default_rng(seed)
    ndim = len(dims)
    ks = _ball_vectors(rng, n_modes, ndim, 4.0)
    amps = rng.uniform(0.5, 1.0, size=n_modes)
    phis = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    X = _unit_grid(dims, coords)
    u = np.zeros(tuple(dims), dtype=np.float64)
    for k, a, p in zip(ks, amps, phis):
        u += a * np.sin(p + sum(2.0 * np.pi * k[d] * X[d] for d in range(ndim)))
    idx = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in dims],
                      indexing="ij", sparse=True)
    p = sum(idx) / np.sqrt(ndim)
    p0 = sum((n - 1) / 2.0 for n in dims) / np.sqrt(ndim)
    u += np.tanh((p - p0) / width_cells)
    return u.astype(dtype)


def multilinear_field(dims, coords=None, seed: int = 7) -> np.ndarray:
    """A random polynomial that is linear in each coordinate separately
    (``sum_S c_S prod_{d in S} x_d``): exactly representable on every grid
    of the hierarchy."""
    rng = np.random.default_rng(seed)
    ndim = len(dims)
    X = _unit_grid(dims, coords)
    u = np.zeros(tuple(dims), dtype=np.float64)
    for mask in range(1 << ndim):
        term = rng.uniform(-1.0, 1.0)
        for d in range(ndim):
            if mask >> d & 1:
                term = term * X[d]
        u = u + term
    return u


def batched_shapes(count: int = 256, seed: int = SEED_BATCHED, lo: int = 33,
                   hi: int = 257, ndim: int = 3):
    """Shapes of the batched workload: each axis drawn from U{lo..hi}, and a
    relative bound drawn from {1e-2, 1e-3, 1e-4} per field."""
    rng = np.random.default_rng(seed)
    shapes = [tuple(int(v) for v in rng.integers(lo, hi + 1, size=ndim))
              for _ in range(count)]
    bounds = [float(b) for b in rng.choice([1e-2, 1e-3, 1e-4], size=count)]
    return shapes, bounds
